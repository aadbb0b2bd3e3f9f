"""Pins of the oracle's readings of the paper where the paper points to
sources that are not in it (Sec. 4.3 reconstruction, the polar-axis boundary,
the floors of Sec. 2 and 4.11) and of its Kerr-Schild signal speeds (Sec. 4.4).

Each check compares the oracle with something other than itself:
  - the polar ghost zones against a smooth Cartesian field written in the
    grid's spherical chart and continued across the axis (theta -> -theta is
    the same point as phi -> phi + pi);
  - the floors against the inequalities they must establish and the
    quantities they must leave alone (the gas velocity u~, the field);
  - the PPM edge values against the exact point values of a parabola and
    against the fourth order of the Colella-Woodward interface formula on
    smooth data (MC alone gives second order), and the monotonicity limiter
    against its defining property;
  - the signal speeds against the textbook relativistic velocity addition in
    the orthonormal frame of the normal (ZAMO) observer, mapped to coordinate
    speeds with the lapse and shift, at Kerr-Schild points inside and outside
    the horizon.
No GPU is needed."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

RHO, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3 = range(12)


# ------------------------------------------------------ polar ghost zones ----

def _theta(x2, h):
    return math.pi * x2 + 0.5 * (1.0 - h) * math.sin(2.0 * math.pi * x2)


def _spherical_field(r, th, ph, h):
    """Primitives of a smooth Cartesian field at the chart point (r, th, ph),
    th allowed outside [0, pi]: scalars are functions of (X, Y, Z); vectors
    are Cartesian vector fields expressed in the coordinate basis of
    (r, theta, phi) and then of the internal chart (x1 = ln r, x2, x3)."""
    st, ct, sp, cp = math.sin(th), math.cos(th), math.sin(ph), math.cos(ph)
    X, Y, Z = r * st * cp, r * st * sp, r * ct
    e_r = np.array([st * cp, st * sp, ct])
    e_t = r * np.array([ct * cp, ct * sp, -st])
    e_p = r * st * np.array([-sp, cp, 0.0])

    def comps(V, x2):
        # contravariant (r, theta, phi) components, then divided by the map's
        # dr/dx1 = r, dtheta/dx2, dphi/dx3 = 2 pi
        j2 = math.pi * (1.0 + (1.0 - h) * math.cos(2.0 * math.pi * x2))
        return np.array([V @ e_r / r, V @ e_t / (r * r) / j2, V @ e_p / (r * r * st * st) / (2 * math.pi)])

    P = np.zeros(12)
    P[RHO] = 1.0 + 0.01 * X + 0.02 * Y + 0.003 * Z * Z
    P[UU] = 0.5 + 0.001 * X * Y + 0.01 * Z
    P[ER] = 2.0 + 0.02 * X - 0.01 * Y + 0.005 * Z
    vel = np.array([0.1 + 0.01 * Y, -0.07 + 0.02 * X, 0.2 + 0.01 * Z])
    fld = np.array([0.03 * Z, 0.05 + 0.01 * X, 1.0 - 0.02 * Y])
    vrad = np.array([-0.2 + 0.01 * Z, 0.1 * math.sin(0.1 * X), 0.05 + 0.01 * Y])
    return P, vel, fld, vrad, comps


def _field_prims(r, x2, ph, h):
    th = _theta(x2, h)
    P, vel, fld, vrad, comps = _spherical_field(r, th, ph, h)
    P[U1:U3 + 1] = comps(vel, x2)
    P[B1:B3 + 1] = comps(fld, x2)
    P[UR1:UR3 + 1] = comps(vrad, x2)
    return P


def test_polar_ghosts_continue_a_cartesian_field_across_the_axis():
    """Kerr-Schild chart with a = 0 (spherical polar): every theta ghost zone,
    at both poles and in the phi ghost corners, equals the analytic field at
    the ghost's own centre (theta < 0 or > pi), i.e. the zone half a turn away
    in phi with u~^theta, B^theta, u~^theta_rad negated."""
    h = 0.3
    n = (6, 8, 8)
    cfg = W.base_params()
    cfg.update(metric=1, a_spin=0.0, R0=0.0, hslope=h, n=list(n),
               x0=[math.log(3.0), 0.0, 0.0], dx=[(math.log(10.0) - math.log(3.0)) / n[0], 1.0 / n[1], 1.0 / n[2]],
               bc=[1, 1, 2, 2, 0, 0])
    x1c = [cfg["x0"][0] + (i + 0.5) * cfg["dx"][0] for i in range(n[0])]
    P = np.zeros((12, n[2], n[1], n[0]))
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                P[:, k, j, i] = _field_prims(math.exp(x1c[i]), (j + 0.5) / n[1], 2 * math.pi * (k + 0.5) / n[2], h)
    o = O.Oracle(cfg)
    o.set_prims(P)
    G = o.prims_with_ghosts(fill=True)
    ng = 4
    checked = 0
    for k in range(-ng, n[2] + ng):
        for j in list(range(-ng, 0)) + list(range(n[1], n[1] + ng)):
            for i in range(n[0]):
                x2 = (j + 0.5) / n[1]
                ph = 2 * math.pi * (k + 0.5) / n[2]
                ref = _field_prims(math.exp(x1c[i]), x2, ph, h)
                got = G[:, k + ng, j + ng, i + ng]
                assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max(), (i, j, k, got - ref)
                checked += 1
    assert checked == 2 * ng * (n[2] + 2 * ng) * n[0]


# ------------------------------------------------------------------ floors ----

def _bsq(p, x, P):
    gcov, gcon, _, alpha = O.metric(p, x)
    ut = P[U1:U3 + 1]
    gam = math.sqrt(1.0 + ut @ gcov[1:, 1:] @ ut)
    ucon = np.zeros(4)
    ucon[0] = gam / alpha
    ucon[1:] = ut - gam * alpha * gcon[0, 1:]
    ucov = gcov @ ucon
    B = P[B1:B3 + 1]
    bt = B @ ucov[1:]
    bcon = np.zeros(4)
    bcon[0] = bt
    bcon[1:] = (B + bt * ucon[1:]) / ucon[0]
    return float(bcon @ gcov @ bcon), gam


def _gamma_rad(p, x, P):
    gcov = O.metric(p, x)[0]
    ur = P[UR1:UR3 + 1]
    return math.sqrt(1.0 + ur @ gcov[1:, 1:] @ ur)


def test_floors_establish_their_bounds_and_nothing_else():
    """Sec. 2 and the torus set-up (Sec. 6): rho0 >= f_rho r^p_rho, b^2/rho0 <=
    200, u_g/rho0 <= 1e10, u_g >= f_u r^p_u, b^2/u_g <= 1e5, gamma_gas <= 50,
    gamma_rad <= 100, Ebar > 0.  After the floors every bound holds; a value
    that changed sits on its bound (to round-off); the floors raise rho0 and u_g at
    fixed gas velocity u~ (only the Lorentz-factor cap rescales u~, keeping
    its direction) and never touch B; applying them twice changes nothing
    (beyond round-off where a Lorentz-factor cap acted);
    a state inside every bound comes back bit for bit."""
    cfg, _ = W.torus((16, 8, 4), seed=1)
    p = O.make_params(cfg)
    rng = W.rng(2024)
    acted = {"rho": 0, "u": 0, "bsq_rho": 0, "bsq_u": 0, "u_rho": 0, "gam": 0, "gam_rad": 0, "E": 0}
    for trial in range(400):
        x = [0.0, rng.uniform(math.log(1.2), math.log(50.0)), rng.uniform(0.02, 0.98), rng.uniform(0, 1)]
        r = cfg["R0"] + math.exp(x[1])
        P = np.zeros(12)
        P[RHO] = 10 ** rng.uniform(-12, 0)
        P[UU] = 10 ** rng.uniform(-14, 0 if trial % 5 else 4)  # some hot enough for u_g/rho0 > 1e10
        P[U1:U3 + 1] = rng.normal(size=3) * 10 ** rng.uniform(-3, 2.5) / np.array([r, 3.0, 6.0])
        P[B1:B3 + 1] = rng.normal(size=3) * 10 ** rng.uniform(-6, -1) / np.array([r, 3.0, 6.0])
        P[ER] = 10 ** rng.uniform(-10, 0) * (1 if trial % 7 else -1)
        P[UR1:UR3 + 1] = rng.normal(size=3) * 10 ** rng.uniform(-2, 3) / np.array([r, 3.0, 6.0])
        Q = O.apply_floors(p, x, P)
        bsq, gam = _bsq(p, x, Q)
        bsq0, gam0 = _bsq(p, x, P)
        grad0, grad = _gamma_rad(p, x, P), _gamma_rad(p, x, Q)
        tol = 1e-12
        # Lorentz-factor caps: at fixed direction, exactly on the cap when they act
        if gam0 > cfg["gamma_gas_max"]:
            acted["gam"] += 1
            assert gam == pytest.approx(cfg["gamma_gas_max"], rel=1e-12)
            f = Q[U1:U3 + 1] / P[U1:U3 + 1]
            assert np.allclose(f, f[0], rtol=1e-14) and 0 < f[0] < 1
        else:
            assert np.array_equal(Q[U1:U3 + 1], P[U1:U3 + 1])
        if grad0 > cfg["gamma_rad_max"]:
            acted["gam_rad"] += 1
            assert grad == pytest.approx(cfg["gamma_rad_max"], rel=1e-12)
        else:
            assert np.array_equal(Q[UR1:UR3 + 1], P[UR1:UR3 + 1])
        assert np.array_equal(Q[B1:B3 + 1], P[B1:B3 + 1])
        # density and energy bounds, with b^2 of the final velocity
        rfl = cfg["floor_rho0"] * r ** cfg["floor_rho_pow"]
        ufl = cfg["floor_u0"] * r ** cfg["floor_u_pow"]
        # b^2 = b^mu b_mu of a moving state cancels terms of order gamma^2 b^2,
        # so two evaluations of it (the floors' and this test's) agree to about
        # gamma^2 eps (gamma <= 50 after the cap): its bounds get that tolerance
        tb = max(tol, 10.0 * gam * gam * 2.220446049250313e-16)
        assert Q[RHO] >= rfl * (1 - tol) and Q[RHO] >= bsq / cfg["bsq_rho_max"] * (1 - tb)
        assert Q[UU] >= ufl * (1 - tol) and Q[UU] >= bsq / cfg["bsq_u_max"] * (1 - tb)
        assert Q[RHO] >= Q[UU] / cfg["u_rho_max"] * (1 - tol)
        assert Q[ER] > 0.0
        if Q[UU] != P[UU]:
            assert Q[UU] > P[UU]
            assert Q[UU] == pytest.approx(max(ufl, bsq / cfg["bsq_u_max"]), rel=max(1e-13, tb))
            acted["u" if ufl >= bsq / cfg["bsq_u_max"] else "bsq_u"] += 1
        if Q[RHO] != P[RHO]:
            assert Q[RHO] > P[RHO]
            bounds = (rfl, bsq / cfg["bsq_rho_max"], Q[UU] / cfg["u_rho_max"])
            assert Q[RHO] == pytest.approx(max(bounds), rel=max(1e-13, tb))
            acted[("rho", "bsq_rho", "u_rho")[int(np.argmax(bounds))]] += 1
        if P[ER] > 0:
            assert Q[ER] == P[ER]
        else:
            acted["E"] += 1
        # idempotent: bit for bit unless a Lorentz-factor cap acted (its
        # rescaled velocity can sit one ulp above the cap, and b^2 at gamma ~ 50
        # amplifies that ulp in the density and energy floors)
        Q2 = O.apply_floors(p, x, Q)
        if gam0 <= cfg["gamma_gas_max"] and grad0 <= cfg["gamma_rad_max"]:
            assert np.array_equal(Q2, Q)
        else:
            assert np.allclose(Q2, Q, rtol=1e-10, atol=0.0)
    # every branch was exercised
    assert all(v > 0 for v in acted.values()), str(acted)
    # a state inside every bound is returned bit for bit
    x = [0.0, math.log(10.0), 0.4, 0.3]
    P = np.zeros(12)
    P[RHO], P[UU], P[ER] = 1.0, 0.1, 0.3
    P[U1:U3 + 1] = [0.01, 0.02, -0.01]
    P[B1:B3 + 1] = [1e-3, 2e-4, 1e-4]
    P[UR1:UR3 + 1] = [0.05, -0.01, 0.02]
    assert np.array_equal(O.apply_floors(p, x, P), P)


# -------------------------------------------------------------------- PPM ----

def _cell_avgs_parabola(xc, h, a, b, c):
    return a + b * xc + c * (xc * xc + h * h / 12.0)


def test_ppm_edges_exact_for_a_parabola():
    """Away from extrema and without flattening, the Colella-Woodward edge
    values of cell averages of a parabola are its point values at the cell
    edges (the interface formula is exact for cubics; MC slopes equal the
    central ones here and the monotonicity limiter does not act)."""
    h = 0.05
    a, b, c = 0.7, 1.0, 0.3
    for i in range(2, 18):
        xc = np.array([(i + m - 2 + 0.5) * h for m in range(5)])
        s = _cell_avgs_parabola(xc, h, a, b, c)
        aL, aR = O.ppm_cell(s, 0.0)
        q = lambda x: a + b * x + c * x * x
        xl, xr = i * h, (i + 1) * h
        assert aL == pytest.approx(q(xl), rel=1e-14, abs=1e-15)
        assert aR == pytest.approx(q(xr), rel=1e-14, abs=1e-15)
    # full flattening: first order (the cell average on both edges)
    aL, aR = O.ppm_cell(s, 1.0)
    assert aL == s[2] and aR == s[2]


def _edge_errors(n, recon):
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    avg = (np.exp(xc + 0.5 * h) - np.exp(xc - 0.5 * h)) / h  # exact cell averages of e^x
    err = 0.0
    for i in range(2, n - 2):
        if recon == "ppm":
            aL, aR = O.ppm_cell(avg[i - 2:i + 3], 0.0)
        else:
            d = O.mc_slope(avg[i - 1], avg[i], avg[i + 1])
            aL, aR = avg[i] - 0.5 * d, avg[i] + 0.5 * d
        err = max(err, abs(aL - math.exp(i * h)), abs(aR - math.exp((i + 1) * h)))
    return err


def test_ppm_edges_fourth_order_mc_second():
    """Smooth monotone data (cell averages of e^x): the PPM edge values
    converge at fourth order (error ratio near 16 per halving of h), the MC
    edge values at second (near 4): a wrong coefficient in the parabola
    would drop PPM to second order."""
    e32, e64 = _edge_errors(32, "ppm"), _edge_errors(64, "ppm")
    m32, m64 = _edge_errors(32, "mc"), _edge_errors(64, "mc")
    assert e32 / e64 > 12.0, (e32, e64)
    assert 3.0 < m32 / m64 < 5.0, (m32, m64)
    assert e64 < 1e-3 * m64


def test_ppm_limiter_monotone_parabola():
    """On random stencils the limited parabola of the centre cell is flat
    (aL = aR = q, at a local extremum) or monotone in the cell: q lies between
    aL and aR and |6 (q - (aL + aR)/2)| <= |aR - aL| (the parabola's extremum
    is not inside the cell)."""
    rng = W.rng(99)
    flat = mono = 0
    for _ in range(2000):
        s = rng.normal(size=5) * 10 ** rng.uniform(-3, 3) + rng.uniform(-1, 1)
        aL, aR = O.ppm_cell(s, 0.0)
        q = s[2]
        if aL == q and aR == q:
            flat += 1
            continue
        mono += 1
        dd = aR - aL
        assert (q - aL) * (aR - q) > 0.0
        assert abs(6.0 * (q - 0.5 * (aL + aR))) <= abs(dd) * (1 + 1e-12)
    assert flat > 100 and mono > 100


# ------------------------------------------------- Kerr-Schild signal speeds ----

def _zamo_speeds(gcov, gcon, ut, c2, d):
    """Coordinate signal speeds along x^d from the textbook velocity addition
    in the normal observer's orthonormal frame: the wave front normal to x^d
    moves at Omega = [V_n (1-c^2) +- c sqrt((1-V^2)(1 - V^2 c^2 - V_n^2 (1-c^2)))]
    / (1 - V^2 c^2) relative to that observer (V the fluid's 3-velocity, V_n
    its component along the unit normal), and v = alpha sqrt(gamma^dd) Omega
    - beta^d in coordinates (lapse alpha, shift beta, inverse spatial metric
    gamma^dd)."""
    alpha = math.sqrt(-1.0 / gcon[0, 0])
    beta_d = -gcon[0, d] / gcon[0, 0]
    gdd_inv = gcon[d, d] - gcon[0, d] ** 2 / gcon[0, 0]
    W2 = 1.0 + ut @ gcov[1:, 1:] @ ut
    lor = math.sqrt(W2)
    V2 = (W2 - 1.0) / W2
    Vn = ut[d - 1] / (lor * math.sqrt(gdd_inv))
    c = math.sqrt(c2)
    root = c * math.sqrt((1.0 - V2) * (1.0 - V2 * c2 - Vn * Vn * (1.0 - c2)))
    om = [(Vn * (1.0 - c2) - root) / (1.0 - V2 * c2), (Vn * (1.0 - c2) + root) / (1.0 - V2 * c2)]
    return [alpha * math.sqrt(gdd_inv) * o - beta_d for o in om]


@pytest.mark.parametrize("kappa", [0.0, 30.0])
def test_kerr_schild_signal_speeds_by_zamo_velocity_addition(kappa):
    """Gas (fast magnetosonic c^2 = c_s^2 + v_A^2 - c_s^2 v_A^2) and radiation
    (c^2 = min(1/3, (4/(3 tau))^2), tau = kappa_tot sqrt(g_dd) dx_d) speeds of
    the oracle at random Kerr-Schild points, r in [1.2, 50] (inside and
    outside the horizon), all three directions, against the 3+1 route."""
    cfg, x, P = W.random_states(300, seed=77, metric=1, gamma_max=5.0, gamma_rad_max=3.0)
    x[::6, 1] = np.log(W.rng(78).uniform(1.2, 1.34, len(x[::6])))  # r inside the horizon r_H = 1.348
    cfg.update(opacity=0, kappa_abs0=kappa, kappa_es0=0.5 * kappa, kappa_scale=1.0)
    p = O.make_params(cfg)
    gam = cfg["gam"]
    inside = 0
    worst = 0.0
    for n in range(len(x)):
        gcov, gcon, _, _ = O.metric(p, x[n])
        inside += gcon[1, 1] < 0
        bsq, _ = _bsq(p, x[n], P[n])
        pg = (gam - 1.0) * P[n][UU]
        w = P[n][RHO] + P[n][UU] + pg
        cs2 = gam * pg / w
        va2 = bsq / (w + bsq)
        c2g = cs2 + va2 - cs2 * va2
        for d in (1, 2, 3):
            _, sp = O.flux(p, x[n], d, P[n])
            vg = _zamo_speeds(gcov, gcon, P[n][U1:U3 + 1], c2g, d)
            tau = 1.5 * kappa * P[n][RHO] * math.sqrt(gcov[d, d]) * cfg["dx"][d - 1]
            c2r = 1.0 / 3.0 if tau == 0.0 else min(1.0 / 3.0, (4.0 / (3.0 * tau)) ** 2)
            vr = _zamo_speeds(gcov, gcon, P[n][UR1:UR3 + 1], c2r, d)
            scale = math.sqrt(max(gcon[d, d] - gcon[0, d] ** 2 / gcon[0, 0], 0.0)) * math.sqrt(-1.0 / gcon[0, 0]) \
                + abs(gcon[0, d] / gcon[0, 0])
            for got, ref in ((sp[0], vg[0]), (sp[1], vg[1]), (sp[2], vr[0]), (sp[3], vr[1])):
                worst = max(worst, abs(got - ref) / scale)
    print("largest speed difference / speed scale: %.2e" % worst)
    assert worst < 1e-10
    assert inside > 5
