"""Pins of the CPU oracle to results fixed by the paper and by the mathematics.

Every check here compares the oracle with something other than itself: a
closed form, a textbook special-relativistic formula, a coordinate
transformation done by hand, an identity of the M1 closure (Sec. 3.1), an
exact scalar root, or a conservation law.  None of these tests needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

RHO, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3 = range(12)
ETA = np.diag([-1.0, 1.0, 1.0, 1.0])


def ks_params(a=0.9375, R0=0.0, h=0.3):
    cfg = W.base_params()
    cfg.update(metric=1, a_spin=a, R0=R0, hslope=h)
    return cfg


def mink_params(**kw):
    cfg = W.base_params()
    cfg.update(kw)
    return cfg


# ---------------------------------------------------------------- metric ----

def test_metric_inverse_and_gdet_closed_form():
    cfg, x, _ = W.random_states(300, seed=11, metric=1)
    p = O.make_params(cfg)
    a, h = cfg["a_spin"], cfg["hslope"]
    for n in range(len(x)):
        gcov, gcon, gdet, alpha = O.metric(p, x[n])
        assert np.abs(gcov @ gcon - np.eye(4)).max() < 1e-12
        r = cfg["R0"] + math.exp(x[n, 1])
        th = math.pi * x[n, 2] + 0.5 * (1 - h) * math.sin(2 * math.pi * x[n, 2])
        Sig = r * r + a * a * math.cos(th) ** 2
        jac = (r - cfg["R0"]) * math.pi * (1 + (1 - h) * math.cos(2 * math.pi * x[n, 2])) * 2 * math.pi
        assert gdet == pytest.approx(Sig * math.sin(th) * jac, rel=1e-12)
        # Kerr-Schild lapse: g^tt = -(1 + 2r/Sigma)
        assert alpha == pytest.approx(1.0 / math.sqrt(1.0 + 2.0 * r / Sig), rel=1e-13)


@pytest.mark.parametrize("a,h", [(0.9375, 0.3), (0.0, 1.0)])
def test_inverse_metric_entries_closed_form(a, h):
    """Every entry of g^{mu nu} against the textbook Kerr-Schild inverse
    (g^tt = -(1 + 2r/S), g^tr = 2r/S, g^rr = Delta/S, g^rphi = a/S,
    g^thth = 1/S, g^phph = 1/(S sin^2 th), S = r^2 + a^2 cos^2 th) divided by
    the internal-coordinate Jacobians J_mu J_nu, each entry to 1e-13 of
    itself, from the horizon out to r = 1e6 (the static atmosphere's radius,
    where the covariant entries span thirteen decades)."""
    p = O.make_params(ks_params(a=a, h=h))
    for r in (1.2, 1.5, 3.0, 15.0, 50.0, 1e4, 1e6, 1.4e6):
        for x2 in (0.07, 0.3, 0.5, 0.77):
            gcov, gcon, gdet, alpha = O.metric(p, [0.0, math.log(r), x2, 0.3])
            th = math.pi * x2 + 0.5 * (1 - h) * math.sin(2 * math.pi * x2)
            S = r * r + a * a * math.cos(th) ** 2
            D = r * r - 2 * r + a * a
            J = [1.0, r, math.pi * (1 + (1 - h) * math.cos(2 * math.pi * x2)), 2 * math.pi]
            ks = np.zeros((4, 4))
            ks[0, 0] = -(1 + 2 * r / S)
            ks[0, 1] = ks[1, 0] = 2 * r / S
            ks[1, 1] = D / S
            ks[1, 3] = ks[3, 1] = a / S
            ks[2, 2] = 1 / S
            ks[3, 3] = 1 / (S * math.sin(th) ** 2)
            want = ks / np.outer(J, J)
            nz = want != 0.0
            err = np.abs(gcon[nz] - want[nz]) / np.abs(want[nz])
            assert err.max() < 1e-13, (r, x2, err.max())
            assert np.all(gcon[~nz] == 0.0) or np.abs(gcon[~nz]).max() < 1e-16 * np.abs(gcon).max()


def test_ks_grr_vanishes_on_horizon():
    # g^{rr} = Delta/Sigma in Kerr-Schild; in code coordinates divided by (dr/dx1)^2.
    a = 0.9375
    p = O.make_params(ks_params(a=a))
    rH = 1.0 + math.sqrt(1.0 - a * a)
    assert rH == pytest.approx(1.348, abs=1e-3)
    for th_x in (0.2, 0.5, 0.8):
        _, gin, _, _ = O.metric(p, [0, math.log(rH), th_x, 0.1])
        assert abs(gin[1, 1]) < 1e-13
        _, gi2, _, _ = O.metric(p, [0, math.log(rH * 0.99), th_x, 0.1])
        _, gi3, _, _ = O.metric(p, [0, math.log(rH * 1.01), th_x, 0.1])
        assert gi2[1, 1] < 0.0 < gi3[1, 1]


# ------------------------------------------------------------ connection ----

def test_connection_schwarzschild_closed_forms():
    """a = 0, R0 = 0: coordinate transformation of textbook Schwarzschild
    Christoffel symbols into the internal (x1, x2, x3) chart."""
    h = 0.3
    p = O.make_params(ks_params(a=0.0, h=h))
    for x1, x2 in ((math.log(3.0), 0.3), (math.log(17.0), 0.61)):
        G = O.connection(p, [0, x1, x2, 0.2])
        th = math.pi * x2 + 0.5 * (1 - h) * math.sin(2 * math.pi * x2)
        thp = math.pi * (1 + (1 - h) * math.cos(2 * math.pi * x2))
        thpp = -2 * math.pi ** 2 * (1 - h) * math.sin(2 * math.pi * x2)
        r = math.exp(x1)
        # Gamma^theta_{r theta} = 1/r  ->  x-chart: (dr/dx1)/r = 1
        assert G[2, 1, 2] == pytest.approx(1.0, rel=1e-12)
        assert G[2, 2, 1] == pytest.approx(1.0, rel=1e-12)
        # pure chart term theta''/theta'
        assert G[2, 2, 2] == pytest.approx(thpp / thp, rel=1e-12, abs=1e-14)
        # Gamma^theta_{phi phi} = -sin cos -> (2 pi)^2/theta' (-sin cos)
        assert G[2, 3, 3] == pytest.approx(-(2 * math.pi) ** 2 * math.sin(th) * math.cos(th) / thp,
                                           rel=1e-12)
        # Gamma^r_{theta theta} = -(r - 2)  ->  theta'^2/r * (-(r-2))
        assert G[1, 2, 2] == pytest.approx(-thp ** 2 * (r - 2.0) / r, rel=1e-12)


def test_connection_metric_compatibility():
    """nabla_k g_{mn} = 0 with d_k g from 4th-order differences of the metric."""
    cfg, x, _ = W.random_states(20, seed=5, metric=1)
    p = O.make_params(cfg)
    for n in range(len(x)):
        G = O.connection(p, x[n])
        g0, _, _, _ = O.metric(p, x[n])
        dg = np.zeros((4, 4, 4))
        for k in (1, 2):
            hh = 1e-3
            vals = []
            for s in (-2, -1, 1, 2):
                xx = x[n].copy()
                xx[k] += s * hh
                vals.append(O.metric(p, xx)[0])
            dg[k] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * hh)
        cov = dg - np.einsum("lkm,ln->kmn", G, g0) - np.einsum("lkn,ml->kmn", G, g0)
        assert np.abs(cov).max() < 1e-7 * max(1.0, np.abs(g0).max())


def test_killing_sources_vanish_in_kerr_schild():
    """Stationary, axisymmetric metric: SM_t = SM_phi = 0 for any state."""
    cfg, x, P = W.random_states(100, seed=12, metric=1)
    p = O.make_params(cfg)
    for n in range(len(x)):
        U, SM = O.prim_to_cons(p, x[n], P[n])
        scale = np.abs(SM).max() + 1e-300
        for q in (1, 4, 8, 11):
            assert abs(SM[q]) < 1e-10 * scale


# ------------------------------------------- stress tensors, Minkowski textbook

def sr_mhd_tensors(P, gam):
    """Textbook special-relativistic MHD + M1 stress tensors (contravariant)."""
    ut = P[U1:U3 + 1]
    g = math.sqrt(1.0 + ut @ ut)
    v = ut / g
    B = P[B1:B3 + 1]
    b0 = g * (B @ v)
    bi = B / g + b0 * v
    bcon = np.concatenate([[b0], bi])
    bsq = B @ B / g ** 2 + (B @ v) ** 2
    ucon = np.concatenate([[g], ut])
    pg = (gam - 1) * P[UU]
    w = P[RHO] + P[UU] + pg
    Tup = (w + bsq) * np.outer(ucon, ucon) + (pg + 0.5 * bsq) * np.linalg.inv(ETA) - np.outer(bcon, bcon)
    ur = P[UR1:UR3 + 1]
    urc = np.concatenate([[math.sqrt(1.0 + ur @ ur)], ur])
    Rup = (4.0 / 3.0) * P[ER] * np.outer(urc, urc) + (P[ER] / 3.0) * np.linalg.inv(ETA)
    return Tup, Rup, ucon, urc, bsq


def test_minkowski_conserved_and_flux_textbook():
    cfg, x, P = W.random_states(200, seed=21, metric=0)
    p = O.make_params(cfg)
    for n in range(len(x)):
        Tup, Rup, ucon, _, _ = sr_mhd_tensors(P[n], cfg["gam"])
        Tmix = Tup @ ETA
        Rmix = Rup @ ETA
        U, SM = O.prim_to_cons(p, x[n], P[n])
        ref = np.concatenate([[P[n, RHO] * ucon[0], Tmix[0, 0] + P[n, RHO] * ucon[0]], Tmix[0, 1:],
                              P[n, B1:B3 + 1], Rmix[0]])
        sc = np.abs(ref).max()
        assert np.abs(U - ref).max() < 1e-12 * sc
        assert np.abs(SM).max() == 0.0
        for d in (1, 2, 3):
            F, _ = O.flux(p, x[n], d, P[n])
            v = ucon[1:] / ucon[0]
            Bv = P[n, B1:B3 + 1] * v[d - 1] - P[n, B1 + d - 1] * v
            reff = np.concatenate([[P[n, RHO] * ucon[d], Tmix[d, 0] + P[n, RHO] * ucon[d]], Tmix[d, 1:],
                                   Bv, Rmix[d]])
            assert np.abs(F - reff).max() < 1e-12 * max(sc, np.abs(reff).max())


def test_wavespeeds_velocity_addition():
    """Unmagnetised gas moving along x in flat space: v+- = (v +- c)/(1 +- v c)."""
    cfg = mink_params(opacity=0, kappa_abs0=0.0, kappa_es0=0.0)
    p = O.make_params(cfg)
    gam = cfg["gam"]
    for v, ug, vr in ((0.0, 0.1, 0.0), (0.6, 0.01, -0.3), (-0.9, 3.0, 0.95)):
        P = np.zeros(12)
        P[RHO] = 1.0
        P[UU] = ug
        g = 1 / math.sqrt(1 - v * v)
        P[U1] = g * v
        P[ER] = 1.0
        gr = 1 / math.sqrt(1 - vr * vr)
        P[UR1] = gr * vr
        _, sp = O.flux(p, [0, 0.5, 0.5, 0.5], 1, P)
        pg = (gam - 1) * ug
        cs = math.sqrt(gam * pg / (1 + ug + pg))
        assert sp[1] == pytest.approx((v + cs) / (1 + v * cs), rel=1e-12)
        assert sp[0] == pytest.approx((v - cs) / (1 - v * cs), rel=1e-12)
        c = 1 / math.sqrt(3)
        assert sp[3] == pytest.approx((vr + c) / (1 + vr * c), rel=1e-12)
        assert sp[2] == pytest.approx((vr - c) / (1 - vr * c), rel=1e-12)


# --------------------------------------------------------- M1 closure pins ----

def boost_to(u):
    """Lorentz boost taking contravariant lab components to the rest frame of u."""
    g = u[0]
    v = u[1:] / g
    v2 = v @ v
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = -g * v
    L[1:, 0] = -g * v
    if v2 > 0:
        L[1:, 1:] += (g - 1) * np.outer(v, v) / v2
    return L


def test_levermore_limits():
    assert O.levermore_xi(0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert O.levermore_xi(1.0) == pytest.approx(1.0, rel=1e-15)


def test_m1_tensor_matches_levermore_closure():
    """R^{mu nu} from Eq. Rlab, boosted to the gas frame, has the Levermore
    pressure tensor P^ij = ((1-xi)/2 delta + (3 xi-1)/2 n n) E with
    f = |F|/E (Sec. 3.1)."""
    cfg, x, P = W.random_states(200, seed=31, metric=0)
    p = O.make_params(cfg)
    for n in range(len(x)):
        T, R = O.stress(p, x[n], P[n])
        Rup = R @ np.linalg.inv(ETA)  # R^{mu nu} = R^mu_a eta^{a nu}
        _, _, ucon, _, _ = sr_mhd_tensors(P[n], cfg["gam"])
        L = boost_to(ucon)
        Rh = L @ Rup @ L.T
        E = Rh[0, 0]
        F = Rh[0, 1:]
        f = np.linalg.norm(F) / E
        xi = O.levermore_xi(f)
        nn = F / np.linalg.norm(F)
        Pref = E * (0.5 * (1 - xi) * np.eye(3) + 0.5 * (3 * xi - 1) * np.outer(nn, nn))
        assert np.abs(Rh[1:, 1:] - Pref).max() < 1e-9 * E
        assert np.allclose(Rh[1:, 1:], Rh[1:, 1:].T, rtol=0, atol=1e-12 * E)


def test_four_force_fluid_frame_form():
    """Eq. Gcov boosted to the gas frame gives Eq. Gff:
    G^ = (kappa_abs E^ - lambda, kappa_tot F^i)."""
    cfg, x, P = W.random_states(200, seed=41, metric=0)
    cfg.update(kappa_abs0=0.7, kappa_es0=1.9)
    p = O.make_params(cfg)
    for n in range(len(x)):
        Gcov = O.four_force(p, x[n], P[n])
        Gcon = np.linalg.inv(ETA) @ Gcov
        T, R = O.stress(p, x[n], P[n])
        Rup = R @ np.linalg.inv(ETA)
        _, _, ucon, _, _ = sr_mhd_tensors(P[n], cfg["gam"])
        L = boost_to(ucon)
        Gh = L @ Gcon
        Rh = L @ Rup @ L.T
        rho = P[n, RHO]
        Tg = (cfg["gam"] - 1) * P[n, UU] / rho
        ka, ks = 0.7 * rho, 1.9 * rho
        lam = ka * cfg["a_rad"] * Tg ** 4
        sc = (ka + ks) * abs(Rh[0, 0]) + lam
        assert abs(Gh[0] - (ka * Rh[0, 0] - lam)) < 1e-9 * sc
        assert np.abs(Gh[1:] - (ka + ks) * Rh[0, 1:]).max() < 1e-9 * sc


# ------------------------------------------------------------- inversions ----

@pytest.mark.parametrize("metric", [0, 1])
def test_gas_inversion_round_trip(metric):
    """prim -> cons -> prim through Eq. EMHD / Wprime / vsqeq / tveq.  The
    forward error must stay within the conditioning of the map U -> P:
    u_g is recovered from energy minus rest mass, so its relative error is
    bounded by eps times the condition number kappa = max_q |d ln P / d ln U_q|,
    estimated here by relative perturbations of U of 1e-7."""
    cfg, x, P = W.random_states(300, seed=51 + metric, metric=metric)
    p = O.make_params(cfg)
    eps = np.finfo(float).eps
    checked = 0
    for n in range(len(x)):
        U, _ = O.prim_to_cons(p, x[n], P[n])
        out, rc = O.gas_invert(p, x[n], U, P[n] * 1.05, 1e-15)
        assert rc == 0
        kap = np.ones(5)
        for q in range(8):
            if U[q] == 0.0:
                continue
            Up = U.copy()
            Up[q] *= 1.0 + 1e-7
            o2, rc2 = O.gas_invert(p, x[n], Up, P[n], 1e-15)
            if rc2 != 0:  # a 1e-7 change leaves the admissible set: no bound
                kap[:] = np.inf
                break
            sens = np.abs(o2[:5] - out[:5]) / 1e-7
            kap[:2] = np.maximum(kap[:2], sens[:2] / np.abs(out[:2]))
            kap[2:] = np.maximum(kap[2:], sens[2:] / max(1.0, np.abs(out[2:5]).max()))
        checked += np.isfinite(kap).all()
        assert abs(out[RHO] / P[n, RHO] - 1) < 50 * eps * kap[0]
        assert abs(out[UU] / P[n, UU] - 1) < 50 * eps * kap[1]
        vs = max(1.0, np.abs(P[n, U1:U3 + 1]).max())
        assert np.abs(out[U1:U3 + 1] - P[n, U1:U3 + 1]).max() < 50 * eps * kap[2:].max() * vs
    assert checked > 0.9 * len(x)


@pytest.mark.parametrize("metric", [0, 1])
def test_rad_inversion_round_trip(metric):
    """Closed-form M1 inversion (Eqs. prsol, tvrsol, gammarvsy, ysol) inverts
    Eq. Rlab for gamma_rad below the cap."""
    cfg, x, P = W.random_states(300, seed=61 + metric, metric=metric)
    p = O.make_params(cfg)
    for n in range(len(x)):
        T, R = O.stress(p, x[n], P[n])
        for lim in (0, 2):
            out, neg = O.rad_invert(p, x[n], R[0], lim)
            assert neg == 0
            assert out[0] == pytest.approx(P[n, ER], rel=1e-11)
            gcov, _, _, _ = O.metric(p, x[n])
            ur = P[n, UR1:UR3 + 1]
            scl = math.sqrt(1 + ur @ gcov[1:, 1:] @ ur) / math.sqrt(min(np.diag(gcov)[1:]))
            assert np.abs(out[1:] - ur).max() < 1e-10 * scl


def test_rad_inversion_limiters():
    p = O.make_params(mink_params(gamma_rad_max=100.0))
    x = [0, 0.5, 0.5, 0.5]
    # negative energy: BASIC gives the 1e-300 floor at rest, TYPE2 keeps the momentum
    Rt = np.array([+0.5, 0.2, 0.0, 0.0])  # R^t_t > 0 -> E_rad < 0
    out, neg = O.rad_invert(p, x, Rt, 0)
    assert neg == 1 and out[0] == 1e-300 and np.all(out[1:] == 0)
    out2, neg2 = O.rad_invert(p, x, Rt, 2)
    assert neg2 == 1 and out2[0] > 0
    g2 = 1 + out2[1:] @ out2[1:]
    assert math.sqrt(g2) == pytest.approx(100.0, rel=1e-9)
    # the radiation momentum is kept: R^t_x of the limited state equals 0.2
    P = np.zeros(12)
    P[RHO] = 1
    P[UU] = 1
    P[ER] = out2[0]
    P[UR1:] = out2[1:]
    _, R = O.stress(p, x, P)
    assert R[0, 1] == pytest.approx(0.2, rel=1e-9)
    # superluminal flux with positive energy: BASIC caps gamma at 100
    Rt = np.array([-1.0, 1.5, 0.0, 0.0])
    out3, neg3 = O.rad_invert(p, x, Rt, 0)
    assert neg3 == 0
    assert math.sqrt(1 + out3[1:] @ out3[1:]) == pytest.approx(100.0, rel=1e-9)


# --------------------------------------------------------- implicit solve ----

def scalar_backward_euler(u0, E0, a_rad, gam, rho, kap, h):
    """Exact root of u - u0 = h kappa (E0 + u0 - u - a ((gam-1) u/rho)^4)."""
    f = lambda u: u - u0 - h * kap * ((E0 + u0 - u) - a_rad * ((gam - 1) * u / rho) ** 4)
    lo, hi = 0.0, u0 + E0
    for _ in range(300):
        m = 0.5 * (lo + hi)
        if f(m) > 0:
            hi = m
        else:
            lo = m
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("h,E0", [(1e-3, 0.02), (1e-2, 0.005), (1.0, 0.02), (0.05, 1e-6)])
def test_implicit_uniform_zone_exact(h, E0):
    """A zone at rest in flat space: the implicit stage reduces to one scalar
    equation (energy exchange by absorption/emission), solved by bisection."""
    cfg = mink_params(a_rad=5.0625e6, opacity=0, kappa_abs0=2560.0, kappa_es0=0.4)
    p = O.make_params(cfg)
    x = [0, 0.5, 0.5, 0.5]
    P = np.zeros(12)
    P[RHO] = 1.0
    P[UU] = 0.01
    P[ER] = E0
    U, _ = O.prim_to_cons(p, x, P)
    out, info = O.implicit_zone(p, x, U, P, h)
    ue = scalar_backward_euler(0.01, E0, 5.0625e6, 5 / 3, 1.0, 2560.0, h)
    assert info.method == O.OK_PMHD
    assert out[UU] == pytest.approx(ue, rel=1e-10)
    assert out[ER] == pytest.approx(0.01 + E0 - ue, rel=1e-10)
    assert np.abs(out[U1:U3 + 1]).max() < 1e-14
    assert np.abs(out[UR1:UR3 + 1]).max() < 1e-14


@pytest.mark.parametrize("metric", [0, 1])
def test_implicit_conserves_and_converges(metric):
    """rho0 u^t and B unchanged, gas+radiation energy-momentum conserved
    (Sec. 4.7), and the error function small at the accepted root."""
    cfg, x, P = W.random_states(60, seed=71 + metric, metric=metric, gamma_max=5.0)
    cfg.update(kappa_abs0=3.0, kappa_es0=1.0)
    p = O.make_params(cfg)
    g = W.rng(99)
    nok = 0
    for n in range(len(x)):
        U, _ = O.prim_to_cons(p, x[n], P[n])
        Ps = P[n].copy()
        Ps[UU] *= 1.0 + 0.3 * g.uniform(-1, 1)
        Ps[ER] *= 1.0 + 0.3 * g.uniform(-1, 1)
        h = 10 ** g.uniform(-3, 0)
        out, info = O.implicit_zone(p, x[n], U, Ps, h)
        if info.method == O.BACKUP or info.neg_erad:
            continue
        nok += 1
        U2, _ = O.prim_to_cons(p, x[n], out)
        assert U2[0] == pytest.approx(U[0], rel=1e-12)
        assert np.allclose(U2[5:8], U[5:8], rtol=1e-13, atol=0)
        tot = U[1:5] + U[8:12]
        tot2 = U2[1:5] + U2[8:12]
        sc = np.abs(U[1:5]).max() + np.abs(U[8:12]).max()
        assert np.abs(tot2 - tot).max() < 1e-9 * sc
        assert info.e_T < 1e-9
    assert nok > 40


# ------------------------------------------------------------ grid pins ----

def test_uniform_box_relaxes_to_closed_form_equilibrium():
    """Uniform periodic box: every flux difference vanishes, the total
    u_g + Ebar is conserved and the stiff coupling drives the gas and the
    radiation to Ebar = a T^4 (quartic root by bisection)."""
    cfg, P = W.relax_box(n1=32, perturb=0.0)
    o = O.Oracle(cfg)
    o.set_prims(P)
    for _ in range(6):
        o.step(0.0)
    Q = o.get_prims()
    a, gam = cfg["a_rad"], cfg["gam"]
    tot = P[UU].mean() + P[ER].mean()
    lo, hi = 0.0, 1.0
    for _ in range(300):
        m = 0.5 * (lo + hi)
        if m / (gam - 1) + a * m ** 4 > tot:
            hi = m
        else:
            lo = m
    Teq = 0.5 * (lo + hi)
    assert np.allclose(Q[UU], Teq / (gam - 1), rtol=1e-12, atol=0)
    assert np.allclose(Q[ER], a * Teq ** 4, rtol=1e-12, atol=0)
    assert np.abs(Q[U1:U3 + 1]).max() == 0.0


def test_opacity_field_reduces_to_constant_opacity():
    """Opacity mode 2 (per-zone field K, kappa_abs = K per length) on the
    uniform relaxation box, where rho0 stays 1 in every zone: with
    K = kappa_abs0 * rho0 the run equals the constant-opacity run (mode 0)
    bit for bit, and so reaches the closed-form equilibrium pinned above."""
    cfg, P = W.relax_box(n1=32, perturb=0.0)
    cfg2 = dict(cfg, opacity=W.OPAC_FIELD)
    a, b = O.Oracle(cfg), O.Oracle(cfg2)
    a.set_prims(P)
    b.set_prims(P)
    b.set_opacity_field(np.full(P.shape[1:], cfg["kappa_abs0"] * 1.0))
    for _ in range(4):
        a.step(0.0)
        b.step(0.0)
    assert np.array_equal(a.get_prims(), b.get_prims())


def mirror_x1(A, vector_planes=(U1, B1, UR1)):
    """Reflect a [q, k, j, i] (or [k, j, i]) array across x1 on a periodic
    grid (cell i -> n1-1-i), negating the x1 components of vectors."""
    M = A[..., ::-1].copy()
    if M.ndim == 4:
        for q in vector_planes:
            M[q] *= -1.0
    return M


def test_opacity_field_mirror_symmetry():
    """A periodic Minkowski box with a field, random flow and a strongly
    varying per-zone absorption field, mirrored across x1 (cell i -> n1-1-i,
    x1 components of u, B, u_rad negated, K mirrored), gives the mirrored
    result after one step.  A face state that took the absorption of the
    wrong neighbour, or a field shifted against the primitives, breaks the
    symmetry."""
    cfg, P = W.minkowski_box(n=(8, 6, 5), seed=11, B_amp=0.05)
    cfg = dict(cfg, opacity=W.OPAC_FIELD)
    g = W.rng(5)
    K = np.exp(g.uniform(np.log(1e-2), np.log(1e3), P.shape[1:])) / cfg["dx"][0]
    a, b = O.Oracle(cfg), O.Oracle(cfg)
    a.set_prims(P)
    a.set_opacity_field(K)
    b.set_prims(mirror_x1(P))
    b.set_opacity_field(mirror_x1(K))
    dt = a.cfl_dt()
    assert b.cfl_dt() == pytest.approx(dt, rel=1e-14)
    a.step(dt)
    b.step(dt)
    A, B = a.get_prims(), mirror_x1(b.get_prims())
    for q in range(12):
        sc = np.abs(A[q]).max() + 1e-300
        assert np.abs(A[q] - B[q]).max() <= 1e-10 * sc, q
    # and the field matters: without it (K = 0) the result is different
    c = O.Oracle(cfg)
    c.set_prims(P)
    c.step(dt)
    assert np.abs(c.get_prims()[ER] - A[ER]).max() > 1e-6 * np.abs(A[ER]).max()


def corner_divb(P, dx):
    B = P[B1:B3 + 1]
    out = 0.0
    axes = (3, 2, 1)  # array axes of x1, x2, x3 in [q, k, j, i] -> per component
    div = np.zeros(P.shape[1:])
    for d in range(3):
        b = B[d]
        ax = [2, 1, 0][d]  # axis in [k, j, i]
        t = b - np.roll(b, 1, axis=ax)
        for o in range(3):
            if o == d:
                continue
            t = t + np.roll(t, 1, axis=[2, 1, 0][o])
        div += t / (4.0 * dx[d])
    del out, axes
    return div


def test_periodic_box_conservation_and_divb():
    """Periodic Minkowski box: total mass, gas+radiation energy-momentum and
    magnetic flux conserved to round-off; flux-CT keeps the corner-centred
    divergence of B unchanged."""
    cfg, P = W.minkowski_box(n=(8, 8, 8), seed=3)
    o = O.Oracle(cfg)
    o.set_prims(P)
    p = O.make_params(cfg)

    def totals():
        Q = o.get_prims()
        tot = np.zeros(12)
        for k in range(8):
            for j in range(8):
                for i in range(8):
                    U, _ = O.prim_to_cons(p, [0, 0.5, 0.5, 0.5], Q[:, k, j, i])
                    tot += U
        return tot, Q

    t0, Q0 = totals()
    d0 = corner_divb(Q0, cfg["dx"])
    o.step(0.0)
    assert o.counts()["backup"] == 0
    t1, Q1 = totals()
    d1 = corner_divb(Q1, cfg["dx"])
    e0 = t0[1:5] + t0[8:12]
    e1 = t1[1:5] + t1[8:12]
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    assert np.abs(e1 - e0).max() < 1e-12 * np.abs(e0).max() * 10
    assert np.abs(t1[5:8] - t0[5:8]).max() < 1e-13 * np.abs(Q0[B1:B3 + 1]).sum()
    bsc = np.abs(Q0[B1:B3 + 1]).max() / min(cfg["dx"])
    assert np.abs(d1 - d0).max() < 1e-12 * bsc


def test_beam_front_moves_at_c():
    """Optically thin limit: a radiation beam with gamma_rad = 10 streaming
    into a radiation-free region keeps its front at x0 + c t (Sec. 5.3)."""
    n = 100
    cfg = W.base_params()
    cfg.update(n=[n, 1, 1], dx=[1.0 / n, 1, 1], bc=[1, 1, 0, 0, 0, 0], opacity=0,
               kappa_abs0=0.0, kappa_es0=0.0, courant=0.5)
    P = np.zeros((12, 1, 1, n))
    xc = (np.arange(n) + 0.5) / n
    P[RHO] = 1.0
    P[UU] = 1e-3
    left = xc < 0.3
    P[ER] = np.where(left, 1.0, 1e-8)
    P[UR1] = np.where(left, math.sqrt(99.0), 0.0)
    o = O.Oracle(cfg)
    o.set_prims(P)
    t = 0.0
    while t < 0.4 - 1e-12:
        dt = min(o.cfl_dt(), 0.4 - t)
        o.step(dt)
        t += dt
    Q = o.get_prims()
    # lab-frame energy density -R^t_t = Ebar (4/3 gamma^2 - 1/3)
    g2 = 1 + Q[UR1, 0, 0] ** 2
    Elab = Q[ER, 0, 0] * (4.0 / 3.0 * g2 - 1.0 / 3.0)
    E0 = 1.0 * (4.0 / 3.0 * 100.0 - 1.0 / 3.0)
    front = xc[np.nonzero(Elab > 0.5 * E0)[0].max()]
    assert abs(front - (0.3 + 0.4)) < 2.5 / n


def test_contact_advection_converges():
    """Pressure-balanced density wave advected at v = 0.5 through a periodic
    box: the hyperbolic part (reconstruction, LAXF, RK3) converges to the
    translated profile at better than first order."""
    errs = []
    for n in (32, 64):
        cfg = W.base_params()
        cfg.update(n=[n, 1, 1], dx=[1.0 / n, 1, 1], opacity=0, kappa_abs0=0.0, kappa_es0=0.0,
                   a_rad=1.0)
        xc = (np.arange(n) + 0.5) / n
        v = 0.5
        P = np.zeros((12, 1, 1, n))
        P[RHO] = 1.0 + 0.2 * np.sin(2 * np.pi * xc)
        P[UU] = 0.1
        P[U1] = v / math.sqrt(1 - v * v)
        P[ER] = 1e-12
        P[UR1] = P[U1]
        o = O.Oracle(cfg)
        o.set_prims(P)
        T = 0.4
        t = 0.0
        while t < T - 1e-14:
            dt = min(o.cfl_dt(), T - t)
            o.step(dt)
            t += dt
        Q = o.get_prims()
        exact = 1.0 + 0.2 * np.sin(2 * np.pi * (xc - v * T))
        errs.append(np.abs(Q[RHO, 0, 0] - exact).mean())
    assert errs[0] < 2e-3
    assert errs[0] / errs[1] > 3.0


def test_error_norm_sees_momentum_inside_horizon():
    """Inside the horizon g^{rr} < 0; the merged spatial error norm (Sec. 4.8)
    must still weigh the momentum rows, so a pure theta-momentum perturbation
    of size delta raises e_T at first order in delta."""
    cfg = ks_params()
    cfg.update(kappa_abs0=1.0, kappa_es0=0.4, a_rad=1.0)
    p = O.make_params(cfg)
    x = [0.0, math.log(1.25), 0.43, 0.1]
    P = np.zeros(12)
    P[RHO], P[UU], P[ER] = 1.0, 0.05, 0.02
    P[U1], P[U2], P[U3] = -0.3, 0.01, 0.02
    P[B1], P[B2] = 0.01, 0.002
    U, _ = O.prim_to_cons(p, x, P)
    base = [P[UU], P[U1], P[U2], P[U3]]
    _, e0, _ = O.pmhd_residual(p, x, U, 0.0, base)
    assert e0 < 1e-13
    for delta in (1e-4, 1e-6):
        xg = list(base)
        xg[2] += delta * 0.01
        _, e1, _ = O.pmhd_residual(p, x, U, 0.0, xg)
        assert math.isfinite(e1) and e1 > 1e-3 * delta
