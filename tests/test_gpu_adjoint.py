"""Hand-written reverse mode (lbm_adjoint): dL/dG_w of the contact-angle loss
against central finite differences of the same loss, on the GPU forward and
on the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lattice(nx, ny, gw_field, fsi, drop, **over):
    import paper_1410_2569_gb300 as lbm
    lat = lbm.Lattice.single(nx, ny, lbm.default_params(**over), inputs.flat_walls(nx, ny), fsi,
                             gw_field)
    lat.init_droplet(*drop)
    return lat


def _loss_gpu(nx, ny, gw_field, fsi, drop, T, target, **over):
    lat = _lattice(nx, ny, gw_field, fsi, drop, **over)
    L, th, _ = lat.adjoint(T, target, 0.5, drop[0], 3.0, want_grad=False)
    d = lat.diagnostics(y_w=0.5, x_ref=drop[0])
    return L, d["n_contour"]


def _central_difference(nx, ny, g, x, fsi, drop, T, target, h, **over):
    """(L(g + h e_x) - L(g - h e_x)) / 2h.  The loss is only piecewise smooth:
    the EOS of Eq. (15) has kinks at rho_1 and rho_2, and a node whose density
    passes one of them at some step under the perturbation puts a kink inside
    [-h, h].  Where the differences at h and h/10 disagree, the one at h/10
    (kink outside its interval) is returned."""
    def fd(hh):
        gp, gm = g.copy(), g.copy()
        gp[0, x] += hh
        gm[0, x] -= hh
        Lp, np_ = _loss_gpu(nx, ny, gp, fsi, drop, T, target, **over)
        Lm, nm = _loss_gpu(nx, ny, gm, fsi, drop, T, target, **over)
        assert np_ == nm, "the contour crossing set changed under the perturbation"
        return (Lp - Lm) / (2 * hh)
    a, b = fd(h), fd(h / 10)
    return a if abs(a - b) <= 1e-6 * max(abs(a), 1.0) else b


def _gw_field(nx, ny, value, seed=0):
    rng = np.random.default_rng(seed)
    g = np.zeros((ny, nx))
    g[0, :] = value + 0.02 * rng.standard_normal(nx)  # per-wall-node parameters
    return g


@pytest.mark.parametrize("fsi,gw0,over", [("modified", 0.1, {}), ("density", 0.07, {}),
                                          ("psi", 0.5, {}), ("modified", 0.1, dict(wall="bb")),
                                          ("density", 0.07, dict(ghost="mirror"))])
def test_adjoint_matches_central_differences_gpu(cuda, fsi, gw0, over):
    nx, ny, T, h = 96, 56, 600, 1e-6
    drop = (48.0, 0.5, 16.0, 2.0)
    g = _gw_field(nx, ny, gw0)
    lat = _lattice(nx, ny, g, fsi, drop, **over)
    L0, th0, grad = lat.adjoint(T, 100.0, 0.5, drop[0], 3.0)
    assert np.isfinite(L0) and np.all(np.isfinite(grad))
    assert np.abs(grad[1:-1]).max() == 0.0  # only solid nodes carry G_w
    # nodes under the droplet, near both contact lines and in the vapour
    xs = [48, 40, 31, 33, 62, 64, 70, 20]
    adj = np.array([grad[0, x] for x in xs])
    fds = np.array([_central_difference(nx, ny, g, x, fsi, drop, T, 100.0, h, **over) for x in xs])
    # relative error of the sampled gradient vector (max norm)
    err = np.abs(adj - fds).max() / np.abs(fds).max()
    assert err <= 1e-5, (err, list(zip(xs, adj, fds)))


def test_adjoint_leaves_the_forward_state(cuda):
    nx, ny, T = 64, 40, 300
    drop = (32.0, 0.5, 12.0, 2.0)
    g = _gw_field(nx, ny, 0.1)
    a = _lattice(nx, ny, g, "modified", drop)
    a.adjoint(T, 95.0, 0.5, drop[0], 3.0)
    b = _lattice(nx, ny, g, "modified", drop)
    b.step(T)
    assert a.t == b.t == T
    assert np.array_equal(a.populations(), b.populations())


def test_adjoint_256x128_against_oracle_differences(cuda):
    """256 x 128 lattice, droplet of radius 32, per-wall-node G_w (initially
    uniform 0.1), modified interaction, T = 2000: the gradient on eight
    seeded wall nodes and the contact-line node against central differences
    (h = 1e-6) of the FP64 oracle's own loss, within 1e-5 relative (max
    norm over the sampled nodes)."""
    nx, ny, T, h = 256, 128, 2000, 1e-6
    drop = (128.0, 0.5, 32.0, 2.0)
    g = np.zeros((ny, nx))
    g[0, :] = 0.1
    lat = _lattice(nx, ny, g, "modified", drop)
    L0, th0, grad = lat.adjoint(T, 0.0, 0.5, drop[0], 3.0)  # target filled in below
    target = th0 + 10.0
    lat = _lattice(nx, ny, g, "modified", drop)
    L0, th0b, grad = lat.adjoint(T, target, 0.5, drop[0], 3.0)
    oracle.set_threads(16)

    def oracle_loss(gw):
        o = oracle.Lattice(nx, ny, oracle.paper_params(), inputs.flat_walls(nx, ny), "modified",
                           gw)
        o.init_droplet(*drop)
        o.step(T)
        d = oracle.contact_angle(o.fields()["rho"], inputs.flat_walls(nx, ny), 250.5, 0.5,
                                 drop[0], 3.0)
        return (d["theta_deg"] - target) ** 2, d["n_contour"]
    def oracle_fd(x, hh):
        gp, gm = g.copy(), g.copy()
        gp[0, x] += hh
        gm[0, x] -= hh
        Lp, n1 = oracle_loss(gp)
        Lm, n2 = oracle_loss(gm)
        assert n1 == n2, "the contour crossing set changed under the perturbation"
        return (Lp - Lm) / (2 * hh)
    # eight seeded wall nodes (the configuration's sample) and the node with
    # the largest gradient (a contact line); the differences at h and h/10,
    # the latter where they disagree (a kink of Eq. (15) inside [-h, h])
    rng = np.random.default_rng(4)
    xs = sorted(set(rng.choice(nx, 8, replace=False).tolist())) + [int(np.argmax(np.abs(grad[0])))]
    adj, fds = [], []
    for x in xs:
        a, b = oracle_fd(x, h), oracle_fd(x, h / 10)
        fds.append(a if abs(a - b) <= 1e-6 * max(abs(a), 1.0) else b)
        adj.append(grad[0, x])
    adj, fds = np.array(adj), np.array(fds)
    assert len(xs) == 9
    err = np.abs(adj - fds).max() / np.abs(fds).max()
    assert err <= 1e-5, (err, list(zip(xs, adj, fds)))


def test_autograd_function(cuda):
    import torch

    from paper_1410_2569_gb300.autograd import contact_angle_loss
    nx, ny = 64, 40
    spec = dict(nx=nx, ny=ny, solid=inputs.flat_walls(nx, ny), fsi="modified",
                drop=(32.0, 0.5, 12.0, 2.0), T=200, theta_target=100.0, x_ref=32.0)
    gw = torch.tensor(_gw_field(nx, ny, 0.1), dtype=torch.float64, requires_grad=True)
    loss = contact_angle_loss(gw, spec)
    loss.backward()
    lat = _lattice(nx, ny, gw.detach().numpy(), "modified", spec["drop"])
    L, _, grad = lat.adjoint(200, 100.0, 0.5, 32.0, 3.0)
    assert abs(loss.item() - L) <= 1e-12 * max(1.0, L)
    assert np.allclose(gw.grad.numpy(), grad, rtol=0, atol=1e-12 * np.abs(grad).max())


def test_adjoint_same_gradient_with_block_rows(cuda):
    """The gradient does not depend on the step pipeline: the FP64 warp
    strips (the default) and the block rows step bit-identically, so the
    reverse sweep sees the same forward states."""
    nx, ny, T = 96, 56, 300
    drop = (48.0, 0.5, 16.0, 2.0)
    g = _gw_field(nx, ny, 0.1)
    a = _lattice(nx, ny, g, "modified", drop)
    La, _, ga = a.adjoint(T, 100.0, 0.5, drop[0], 3.0)
    b = _lattice(nx, ny, g, "modified", drop)
    b.set_launch(stages=1)
    Lb, _, gb = b.adjoint(T, 100.0, 0.5, drop[0], 3.0)
    assert La == Lb
    assert np.allclose(ga, gb, rtol=1e-12, atol=1e-14 * np.abs(ga).max())
