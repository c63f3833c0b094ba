"""The dependency lists of the persistent warp strips (lbm_strip_neighbours,
host only, no GPU) against a brute-force construction: item j is listed for
item i exactly when a node of j lies within 4 nodes of a node of i along x
and along y, periodically.  A missing entry would let a strip read
populations a neighbour has not written yet, or overwrite ones it still
reads."""
import ctypes

import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm

ERR_ARG = 1


def _lists(nx, ny, h):
    L = lbm.load()
    n_items, n_nbr = ctypes.c_int(), ctypes.c_int()
    assert L.lbm_strip_neighbours(nx, ny, h, ctypes.byref(n_items), None, None, None, 0,
                                  ctypes.byref(n_nbr)) == 0
    cap = max(3 * n_items.value, n_nbr.value, n_items.value + 1)
    items, off, nbr = (np.zeros(cap, np.int32) for _ in range(3))
    assert L.lbm_strip_neighbours(nx, ny, h, ctypes.byref(n_items), items.ctypes.data,
                                  off.ctypes.data, nbr.ctypes.data, cap,
                                  ctypes.byref(n_nbr)) == 0
    n = n_items.value
    lists = [nbr[off[i]:off[i + 1]].tolist() for i in range(n)]
    return items[:3 * n].reshape(n, 3), lists


def _gap(a0, a1, b0, b1, n):
    """smallest periodic distance between a node of [a0, a1) and one of [b0, b1)"""
    d = np.abs(np.arange(a0, a1)[:, None] - np.arange(b0, b1)[None, :]) % n
    return int(np.minimum(d, n - d).min())


@pytest.mark.parametrize("nx,ny,h", [(64, 40, 7), (33, 20, 2), (400, 200, 30), (130, 48, 1),
                                     (31, 9, 4), (95, 13, 13), (61, 70, 3), (200, 11, 5)])
def test_strip_neighbours_match_brute_force(nx, ny, h):
    items, lists = _lists(nx, ny, h)
    cover = np.zeros((ny, nx), int)
    for x0, y0, y1 in items:
        cover[y0:y1, x0:min(nx, x0 + 30)] += 1
    assert (cover == 1).all()  # the strips tile the lattice once
    for i, (x0, y0, y1) in enumerate(items):
        listed = set(lists[i])
        assert len(listed) == len(lists[i]) and i in listed
        for j, (u0, v0, v1) in enumerate(items):
            near = (_gap(x0, min(nx, x0 + 30), u0, min(nx, u0 + 30), nx) <= 4 and
                    _gap(y0, y1, v0, v1, ny) <= 4)
            assert (j in listed) == near, (i, j)


def test_strip_neighbours_arguments():
    L = lbm.load()
    n, m = ctypes.c_int(), ctypes.c_int()
    assert L.lbm_strip_neighbours(64, 40, 0, ctypes.byref(n), None, None, None, 0,
                                  ctypes.byref(m)) == ERR_ARG
    assert L.lbm_strip_neighbours(2, 40, 4, ctypes.byref(n), None, None, None, 0,
                                  ctypes.byref(m)) == ERR_ARG
    buf = np.zeros(4, np.int32)
    assert L.lbm_strip_neighbours(64, 40, 4, ctypes.byref(n), buf.ctypes.data, buf.ctypes.data,
                                  buf.ctypes.data, 4, ctypes.byref(m)) == ERR_ARG


def _ctx_lists(lat):
    L = lbm.load()
    n_items, n_nbr = ctypes.c_int(), ctypes.c_int()
    assert L.lbm_get_work_items(lat._h, ctypes.byref(n_items), None, None, None, 0,
                                ctypes.byref(n_nbr)) == 0
    n = n_items.value
    cap = max(4 * n, n_nbr.value, n + 1)
    items, off, nbr = (np.zeros(cap, np.int32) for _ in range(3))
    assert L.lbm_get_work_items(lat._h, ctypes.byref(n_items), items.ctypes.data,
                                off.ctypes.data, nbr.ctypes.data, cap, ctypes.byref(n_nbr)) == 0
    return items[:4 * n].reshape(n, 4), [nbr[off[i]:off[i + 1]].tolist() for i in range(n)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [dict(), dict(h=3), dict(h=2, bx=64)])
@pytest.mark.parametrize("widths", ["any", "w4"])
def test_context_lists_of_a_persistent_batch_match_brute_force(cuda, prec, shape, widths):
    """The items and dependency lists a persistent warp-strip batch actually
    runs with (lbm_get_work_items): several instances of uneven sizes (odd
    heights among them), the automatic segment heights and fixed ones; with
    every width a multiple of 4 the FP32 batch runs the column-pair strips
    (60-column items), otherwise the one-row strips (30 columns).  Item j is
    listed for item i exactly when both belong to one instance and a node of
    j lies within 4 nodes of one of i along x and along y (periodic); items
    of other instances are never listed."""
    from paper_1410_2569_gb300 import inputs
    shapes = ([(64, 40), (130, 48), (96, 70), (33, 21), (257, 37)] if widths == "any" else
              [(64, 40), (132, 48), (96, 70), (36, 21), (252, 37)])
    specs = [dict(nx=nx, ny=ny, params=lbm.default_params(prec=prec),
                  solid=inputs.flat_walls(nx, ny), fsi="modified", gw=0.1) for nx, ny in shapes]
    lat = lbm.Lattice(specs)
    lat.set_launch(persistent=True, **shape)
    pipe = lat.launch()["pipeline"]
    assert pipe == (4 if (prec == "fp32" and widths == "w4") else 3)
    W = 60 if pipe == 4 else 30
    items, lists = _ctx_lists(lat)
    for k, (nx, ny) in enumerate(shapes):
        cover = np.zeros((ny, nx), int)
        for inst, x0, y0, y1 in items:
            if inst == k:
                cover[y0:y1, x0:min(nx, x0 + W)] += 1
        assert (cover == 1).all(), k
    heights = {int(y1 - y0) for _, _, y0, y1 in items}
    assert len(heights) > 1  # segments of different heights (odd ny, short last segments)
    for i, (k, x0, y0, y1) in enumerate(items):
        nx, ny = shapes[k]
        listed = set(lists[i])
        assert len(listed) == len(lists[i]) and i in listed
        for j, (kj, u0, v0, v1) in enumerate(items):
            near = (kj == k and _gap(x0, min(nx, x0 + W), u0, min(nx, u0 + W), nx) <= 4 and
                    _gap(y0, y1, v0, v1, ny) <= 4)
            assert (j in listed) == near, (i, j)
    # one launch per step: the same items, no lists
    lat.set_launch()
    items2, lists2 = _ctx_lists(lat)
    assert all(not ls for ls in lists2) and len(items2) > 0
