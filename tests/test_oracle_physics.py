"""Physics pins of the FP64 oracle against the numbers the paper prints
(tests/golden/) and against closed forms: the neutral wall (Sec. III.A),
the G_w -> theta pairs of Figs. 2-4, the Table I ordering of the minimum
densities, flat-interface coexistence against the Maxwell construction of
the printed EOS, the Laplace law, and the spreading exponents of the
dynamic wetting of Sec. III.A (Fig. 7).

The runs are independent and go to a process pool (spawn) at module set-up,
one oracle thread each; the whole module takes about a minute on 8 cores.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
STEPS = 5000  # static angles are within 1 deg of their final value by then


def _table(name):
    rows = []
    for ln in open(os.path.join(GOLD, name)):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            rows.append(ln.split())
    return rows


def _printed_angle(fsi, gw):
    for r in _table("paper_contact_angles.txt"):
        if r[0] == fsi and float(r[1]) == gw:
            return float(r[2])
    raise KeyError((fsi, gw))


# psi-based G_w in this library's units is 3/4 of the printed value (the
# printed Fig. 3 angles are reproduced there; see the design notes)
PSI_SCALE = 0.75

# (interaction, G_w, droplet centre y0, ghost layer of Eq. (7) at the wall,
# wall height y_w for the contact angle)
CASES = {
    "neutral": ("modified", 0.0, 25.5, "copy", 0.5),
    "density+": ("density", 0.07, 0.5, "copy", 0.5),
    "modified+": ("modified", 0.1, 0.5, "copy", 0.5),
    "modified-": ("modified", -0.1, 0.5, "copy", 0.5),
    "psi+": ("psi", 1.0 * PSI_SCALE, 0.5, "copy", 0.5),
    # MIRROR makes the first fluid row the symmetry plane of psi: y_w = 1
    "neutral-mirror": ("modified", 0.0, 1.0, "mirror", 1.0),
}


def _run_sessile(args):
    fsi, gw, y0, ghost, y_w = args
    import oracle
    from paper_1410_2569_gb300 import inputs
    oracle.set_threads(1)
    nx, ny = 300, 100
    solid = inputs.flat_walls(nx, ny)
    o = oracle.Lattice(nx, ny, oracle.paper_params(ghost=ghost), solid, fsi,
                       inputs.wall_gw(solid, gw))
    o.init_droplet(nx / 2, y0, 30.0, 2.0)
    o.step(STEPS)
    return o.diagnostics(y_w, nx / 2, 3.0)


SLAB_SIGMAS = (0.07, 0.084, 0.1, 0.12)


def _run_slab(sigma):
    """A periodic flat slab (liquid between y = 50 and y = 150 of 200 rows),
    uniform along x, to steady state: bulk vapour and liquid densities."""
    import oracle
    oracle.set_threads(1)
    nx, ny = 1, 200
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    d = np.abs(y - ny / 2)
    rho = 1.0 + 0.5 * 499.0 * (1 - np.tanh(2 * (d - 50) / 4.0))
    o = oracle.Lattice(nx, ny, oracle.paper_params(sigma=sigma), np.zeros((ny, nx), np.uint8),
                       "density", 0)
    o.set_density(rho)
    # sigma = 0.084 passes a metastable state (rho_V near 0.98) before it
    # settles between 5e4 and 1e5 steps; the others settle within 5e4
    o.step(120000)
    r = o.fields()["rho"]
    return float(r[ny // 2, 0]), float(r[0, 0])


SPREAD_NX, SPREAD_NY, SPREAD_R, SPREAD_STEPS = 300, 100, 30.0, 1500


def _run_spreading(gw):
    """Spreading radius on the first fluid row every 10 steps; the droplet
    starts half an interface width (2 nodes) above the wall (Sec. III.A)."""
    import oracle
    from paper_1410_2569_gb300 import inputs
    oracle.set_threads(1)
    nx, ny, R = SPREAD_NX, SPREAD_NY, SPREAD_R
    solid = inputs.flat_walls(nx, ny)
    o = oracle.Lattice(nx, ny, oracle.paper_params(), solid, "modified", inputs.wall_gw(solid, gw))
    o.init_droplet(nx / 2, 0.5 + R + 2.0, R, 4.0)
    t, r = [], []
    for k in range(SPREAD_STEPS // 10):
        o.step(10)
        t.append(10 * (k + 1))
        r.append(oracle.contact_radius(o.fields()["rho"], solid, 1, 250.5, nx / 2))
    return np.array(t, float), np.array(r)


def _run_laplace(R):
    import oracle
    oracle.set_threads(1)
    n = 96
    p = oracle.paper_params()
    o = oracle.Lattice(n, n, p, np.zeros((n, n), np.uint8), "density", 0)
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.sqrt((xx - n / 2) ** 2 + (yy - n / 2) ** 2)
    o.set_density(1.0 + 0.5 * 499.0 * (1 - np.tanh(2 * (r - R) / 4.0)))
    o.step(6000)
    rho = o.fields()["rho"]
    dp = oracle.p_eos(p, rho[n // 2, n // 2]) - oracle.p_eos(p, rho[0, 0])
    frac = (rho - rho[0, 0]) / (rho[n // 2, n // 2] - rho[0, 0])
    R_eff = math.sqrt(frac.sum() / math.pi)
    return R_eff, dp


@pytest.fixture(scope="module")
def runs():
    ctx = mp.get_context("spawn")
    spread_gw = [float(r[0]) for r in _table("paper_spreading.txt")]
    jobs = [(_run_sessile, v) for v in CASES.values()] + [(_run_slab, sg) for sg in SLAB_SIGMAS] + \
        [(_run_laplace, R) for R in (14, 18, 22, 26)] + [(_run_spreading, g) for g in spread_gw]
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        handles = [pool.apply_async(f, (a,)) for f, a in jobs]
        out = [h.get(timeout=900) for h in handles]
    k = len(CASES)
    m = k + len(SLAB_SIGMAS)
    return {"sessile": dict(zip(CASES, out[:k])), "slab": dict(zip(SLAB_SIGMAS, out[k:m])),
            "laplace": out[m:m + 4], "spreading": dict(zip(spread_gw, out[m + 4:]))}


def test_neutral_wall_gives_ninety_degrees(runs):
    """G_w = 0: theta = 90 deg analytically, 89.3 deg in the paper (Sec. III.A);
    Table I row 90 deg: rho_min 1.00, rho_max 500.5."""
    d = runs["sessile"]["neutral"]
    assert abs(d["theta_deg"] - 90.0) <= 0.8, d
    assert abs(d["theta_deg"] - _printed_angle("neutral", 0.0)) <= 0.8
    row = [r for r in _table("paper_table1.txt") if r[0] == "90"][0]
    assert abs(d["rho_min"] - float(row[5])) <= 0.02
    assert abs(d["rho_max"] - float(row[6])) <= 0.5


def test_neutral_wall_with_mirror_ghost_gives_ninety_degrees(runs):
    """G_w = 0 with the MIRROR ghost: psi is symmetric about the first fluid
    row, so Eq. (7) sees the droplet and its mirror image and the angle is
    90 deg with y_w on that row (Sec. III.A's analytic value)."""
    d = runs["sessile"]["neutral-mirror"]
    assert abs(d["theta_deg"] - 90.0) <= 0.7, d
    assert d["fit_rms"] < 0.2


@pytest.mark.parametrize("key,printed_gw", [("density+", 0.07), ("modified+", 0.1),
                                            ("modified-", -0.1), ("psi+", 1.0)])
def test_contact_angle_matches_printed_value(runs, key, printed_gw):
    fsi = CASES[key][0]
    d = runs["sessile"][key]
    assert abs(d["theta_deg"] - _printed_angle(fsi, printed_gw)) <= 3.0, d
    assert d["fit_rms"] < 0.2  # a circular cap


def test_theta_increases_with_gw(runs):
    s = runs["sessile"]
    assert s["modified-"]["theta_deg"] < s["neutral"]["theta_deg"] < s["modified+"]["theta_deg"]
    assert s["density+"]["theta_deg"] > 95.0 and s["psi+"]["theta_deg"] > 95.0


def test_table1_ordering_of_rho_min_for_large_angles(runs):
    """For theta > 90 deg the modified interaction keeps the vapour density
    closest to rho_V, the psi-based one deviates most (Table I, Sec. III.B)."""
    s = runs["sessile"]
    rm, rd, rp = (s[k]["rho_min"] for k in ("modified+", "density+", "psi+"))
    assert rm > rd > rp
    assert rp < 0.9 and rm > 0.98


def _p_eos(rho):
    """Eq. (15) with the printed parameters (Sec. III)."""
    cs2 = 1.0 / 3.0
    tV, tM, tL, r1, r2 = 0.64 * cs2, -0.04 * cs2, cs2, 1.36, 481.04
    if rho <= r1:
        return rho * tV
    if rho <= r2:
        return r1 * tV + (rho - r1) * tM
    return r1 * tV + (r2 - r1) * tM + (rho - r2) * tL


def _mechanical_stability(sigma, G=-1.0):
    """Flat-interface coexistence of the continuum model.  In 1-D the normal
    component of the pressure tensor of Eq. (8) is p_EOS + (G/4) psi psi''.
    The sigma term of Eq. (9) gives the e moment a steady non-equilibrium
    part (tau_e - 1/2) S_e = 12 sigma |F_m|^2 / psi^2, i.e. an isotropic
    2 sigma |F_m|^2 / psi^2 = 2 sigma G^2 psi'^2 in the pressure tensor
    (e = -4 rho + 3 tr Pi; sum_a w_a e_a e_a = I).  P_yy = p0 then reads
    p0 - p_EOS = (G/4) psi psi'' + 2 sigma G^2 psi'^2; times psi'/psi^(1+eps)
    the right side is a total derivative for eps = -16 G sigma, so the bulk
    densities obey p_EOS(rho_V) = p_EOS(rho_L) = p0 and
    int_{rho_V}^{rho_L} (p0 - p_EOS) psi' / psi^(1+eps) drho = 0
    (psi' = 0 on the liquid branch of Eq. (15))."""
    from scipy.integrate import quad
    from scipy.optimize import brentq
    cs2 = 1.0 / 3.0
    eps = -16.0 * G * sigma
    psi2 = lambda r: 2.0 * (r * cs2 - _p_eos(r)) / (-G)  # noqa: E731
    r1, r2 = 1.36, 481.04

    def dpsi(r):
        slope = 0.64 * cs2 if r <= r1 else -0.04 * cs2
        return (cs2 - slope) / (-G) / np.sqrt(psi2(r))

    def cond(p0):
        rv = p0 / (0.64 * cs2)
        f = lambda r: (p0 - _p_eos(r)) * dpsi(r) / psi2(r) ** ((1 + eps) / 2)  # noqa: E731
        return quad(f, rv, r2, points=[r1], limit=400)[0]
    p0 = brentq(cond, 0.02, 0.2879)
    rho_L = r2 + (p0 - _p_eos(r2)) / cs2
    return p0 / (0.64 * cs2), rho_L


def test_flat_interface_coexistence_follows_mechanical_stability(runs):
    """Flat-interface coexistence (Sec. II.B).  The paper tunes sigma = 0.084
    for approximate thermodynamic consistency (Maxwell densities of the
    printed EOS: rho_V = 1.0011, rho_L = 499.9975) and prints no
    flat-interface value.  Pinned here, for sigma = 0.07 ... 0.12:
    - mechanical equilibrium of the bulks: p_EOS(rho_V) = p_EOS(rho_L)
      (the momentum flux of a fluid at rest is rho cs^2 + G psi^2 / 2 =
      p_EOS), to 1e-4;
    - the liquid density of the continuum mechanical-stability solution,
      to 1e-4;
    - its vapour density to 5 %: the solution moves by 60 % over this sigma
      range, and the lattice adds a few per cent at an interface four nodes
      wide (an interface along a lattice diagonal settles 4 % higher than
      this one along an axis);
    - the vapour density crosses the Maxwell value between the paper's
      sigma = 0.084 and the continuum's crossing (sigma = 0.092)."""
    rv_by_sigma = {}
    for sigma in SLAB_SIGMAS:
        rl, rv = runs["slab"][sigma]
        pl, pv = _p_eos(rl), _p_eos(rv)
        assert abs(pl - pv) < 1e-4 * pv, (sigma, rl, rv, pl, pv)
        tv, tl = _mechanical_stability(sigma)
        assert abs(rl - tl) / tl < 1e-4, (sigma, rl, tl)
        assert abs(rv / tv - 1.0) < 0.05, (sigma, rv, tv)
        rv_by_sigma[sigma] = rv
    vals = [rv_by_sigma[sg] for sg in SLAB_SIGMAS]
    assert all(a < b for a, b in zip(vals, vals[1:])), vals
    # the sigma at which the slab's vapour reaches the Maxwell density
    s_star = np.interp(1.0011, vals, SLAB_SIGMAS)
    assert 0.084 <= s_star <= 0.0925, s_star


def test_mechanical_stability_solution_pins():
    """The continuum solution itself: sigma -> 0 removes the pressure term
    that stabilises the interface (no coexistence with rho_V > 0 is found
    below eps = 1, the Shan value eps = 0 of Eq. (8) alone gives none), and
    eps = 16 sigma near 1.47 reproduces the Maxwell vapour density."""
    tv, tl = _mechanical_stability(0.0919)
    assert abs(tv - 1.0011) < 0.01 and abs(tl - 499.9975) < 0.05, (tv, tl)
    with pytest.raises(ValueError):
        _mechanical_stability(0.03)


def _laplace_fit(runs):
    R = np.array([r for r, _ in runs["laplace"]])
    dp = np.array([p for _, p in runs["laplace"]])
    A = np.vstack([1 / R, np.ones_like(R)]).T
    (gamma, b), res, *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ np.array([gamma, b])
    r2 = 1 - np.sum((dp - pred) ** 2) / np.sum((dp - dp.mean()) ** 2)
    return gamma, b, r2, dp


def test_laplace_law(runs):
    """2-D Laplace law: dp = gamma / R, a straight line through the origin in
    1/R with positive slope."""
    gamma, b, r2, dp = _laplace_fit(runs)
    assert gamma > 0 and r2 > 0.999, (gamma, b, r2)
    assert abs(b) < 0.1 * dp.min(), (gamma, b, dp)


def test_spreading_exponents(runs):
    """Dynamic wetting (Sec. III.A, Fig. 7): in the inertial regime the
    spreading radius follows r / R = C (t / tau_rho)^n, tau_rho =
    sqrt(rho_L R^3 / gamma), with n = 0.51, 0.485, 0.425 printed for
    theta = 19.0, 69.4, 126.3 deg: n falls as theta rises and is near 1/2
    for small angles.  The fit window t / tau_rho in [0.1, 1] reads "t
    comparable to tau_rho"; gamma comes from the Laplace runs."""
    gamma = _laplace_fit(runs)[0]
    tau = math.sqrt(500.0 * SPREAD_R ** 3 / gamma)
    assert SPREAD_STEPS >= tau, tau
    rows = _table("paper_spreading.txt")
    ns = []
    for r in rows:
        t, rad = runs["spreading"][float(r[0])]
        m = (t >= 0.1 * tau) & (t <= tau)
        assert np.all(rad[m] > 0), rad  # in contact over the whole window
        n, _ = np.polyfit(np.log(t[m] / tau), np.log(rad[m] / SPREAD_R), 1)
        assert abs(n - float(r[2])) <= 0.05, (r, n)
        ns.append(n)
    assert ns[0] > ns[1] > ns[2], ns
