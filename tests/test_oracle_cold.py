"""Pins of the oracle's cold-MHD back-up (Sec. 4.11): when neither the energy
nor the entropy equation gives a solution, a cold, momentum-dominated zone
solves the three momentum equations alone (the reduced 3D PMHD method of
Sec. 4.9) with u_g held at the guess, and the grid step then replaces that
u_g by its neighbours' average.

The cases are flat-space zones without gas-radiation coupling (kappa = 0)
whose explicit gas energy is half the kinetic energy of their motion, so no
u_g >= 0 satisfies the energy equation, and whose radiation is momentum-
dominated (|F| = 4 to 8 E), which no radiation primitives reproduce.  With
kappa = 0 and B = 0 the momentum equations have a closed form:
T^t_i = (rho0 u^t + Gamma u_g u^t) u_i = (D + Gamma u_g gamma) u~_i, so u~ is
parallel to T*_i and its length solves a scalar monotone equation, found here
by bisection."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

RHO, UU, U1, U3, B1, B3, ER, UR1, UR3 = 0, 1, 2, 4, 5, 7, 8, 9, 11
X = [0.0, 0.5, 0.5, 0.5]


def cold_config():
    cfg = W.base_params()
    cfg.update(kappa_abs0=0.0, kappa_es0=0.0)
    return cfg


def cold_cases(count=32, seed=2029, B_amp=0.0):
    """Zones for the cold-MHD back-up: (U*, guess P_s, the true gas state).
    Gas: rho0 log-uniform in [1/e, e], Lorentz factor uniform in [1.01, 1.2]
    (below 11/9, the gas momentum-dominance bound of the cold test) in a random
    direction, u_g = rho0 10^U(-8,-5); U* its conserved state with the energy
    row halved.  Radiation: E = (1 to 3) x the gas kinetic energy
    rho0 gamma (gamma - 1), F = (4 to 8) E in a random direction.  Guess: the
    true gas with u_g scaled by 10^U(-0.3, 0.3) and u~ moved by 0.05 per
    component, radiation E at rest."""
    cfg = cold_config()
    p = O.make_params(cfg)
    g = W.rng(seed)
    out = []
    for _ in range(count):
        rho = math.exp(g.uniform(-1.0, 1.0))
        gam = g.uniform(1.01, 1.2)
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        P = np.zeros(12)
        P[RHO] = rho
        P[UU] = rho * 10.0 ** g.uniform(-8.0, -5.0)
        P[U1:U3 + 1] = d * math.sqrt(gam * gam - 1.0)
        P[B1:B3 + 1] = B_amp * g.uniform(-1.0, 1.0, 3)
        P[ER] = 1e-3 * rho
        U, _ = O.prim_to_cons(p, X, P)
        U[UU] *= 0.5
        E = g.uniform(1.0, 3.0) * rho * gam * (gam - 1.0)
        f = g.standard_normal(3)
        f /= np.linalg.norm(f)
        U[ER] = -E
        U[UR1:UR3 + 1] = g.uniform(4.0, 8.0) * E * f
        Ps = P.copy()
        Ps[UU] = P[UU] * 10.0 ** g.uniform(-0.3, 0.3)
        Ps[U1:U3 + 1] = P[U1:U3 + 1] + 0.05 * g.uniform(-1.0, 1.0, 3)
        Ps[ER] = E
        Ps[UR1:UR3 + 1] = 0.0
        out.append((U, Ps, P))
    return cfg, out


def closed_form_velocity(D, T, gam_ad, ug):
    """u~ with (D + Gamma u_g sqrt(1 + |u~|^2)) u~ = T (flat space, B = 0)."""
    t = np.linalg.norm(T)
    lo, hi = 0.0, t / D
    for _ in range(200):
        m = 0.5 * (lo + hi)
        if (D + gam_ad * ug * math.sqrt(1.0 + m * m)) * m < t:
            lo = m
        else:
            hi = m
    return 0.5 * (lo + hi) * T / t


def test_cold_test_thresholds():
    """The three conditions of the cold test at their closed-form thresholds
    (flat space): u_g = 0.1 rho0 |u~|^2; for a cold gas, (gamma - 1)^2 =
    0.1 (gamma^2 - 1), i.e. gamma = 11/9; for the radiation, |F| = sqrt(10) E.
    Each is crossed by a relative 1e-6 with the other two held inside."""
    cfg = cold_config()
    p = O.make_params(cfg)

    def case(ug_fac=0.5, gam=1.1, fe=5.0, rad_first=False):
        P = np.zeros(12)
        P[RHO] = 1.0
        u = math.sqrt(gam * gam - 1.0)
        P[U1] = u
        P[UU] = 1e-14
        U, _ = O.prim_to_cons(p, X, P)
        Ps = P.copy()
        Ps[UU] = ug_fac * 0.1 * u * u
        U[ER] = -1.0
        U[UR1] = fe
        return O.cold_allowed(p, X, U, Ps)

    assert case() and case(ug_fac=1.0 - 1e-6) and not case(ug_fac=1.0 + 1e-6)
    assert case(gam=11.0 / 9.0 * (1.0 - 1e-6)) and not case(gam=11.0 / 9.0 * (1.0 + 1e-6))
    r10 = math.sqrt(10.0)
    assert case(fe=r10 * (1.0 + 1e-6)) and not case(fe=r10 * (1.0 - 1e-6))


def test_cold_solution_closed_form():
    """Without the explicit entropy (the IMEX case) every zone ends in the
    cold-MHD equations, with u_g exactly the guess's, rho0 u^t conserved, the
    velocity of the closed form to 1e-12, the radiation momentum of U* kept
    (the TYPE2 limiter raises the energy only) and e_T below 1e-12."""
    cfg, cases = cold_cases()
    p = O.make_params(cfg)
    gam_ad = cfg["gam"]
    worst = 0.0
    for U, Ps, _ in cases:
        out, info = O.implicit_zone(p, X, U, Ps, 0.1)
        assert info.cold == 1 and info.entropy == 0 and info.method == O.OK_URAD, (info.method, info.e_T)
        assert info.e_T < 1e-12
        assert out[UU] == Ps[UU]
        Uo, _ = O.prim_to_cons(p, X, out)
        assert Uo[RHO] == pytest.approx(U[RHO], rel=1e-14)
        ut = closed_form_velocity(U[RHO], U[U1:U3 + 1], gam_ad, Ps[UU])
        worst = max(worst, np.abs(out[U1:U3 + 1] - ut).max() / np.linalg.norm(ut))
        assert np.allclose(Uo[UR1:UR3 + 1], U[UR1:UR3 + 1], rtol=1e-12, atol=0.0)
        assert -Uo[ER] > -U[ER]
    print("cold-MHD velocity against the closed form: worst relative error %.2e" % worst)
    assert worst < 1e-12


def test_cold_order_and_conditions():
    """The back-up order of Sec. 4.11: with the explicit entropy of the true
    state the entropy equation solves the zone (it comes first, although the
    zone passes the cold test); without an explicit entropy (not finite) the
    cold-MHD equations do; a zone whose radiation is not momentum-dominated
    (|F| = 2 E) fails the cold test and takes the neighbour-average back-up.
    (An entropy that no u_g > 0 reaches does not make the entropy equation
    fail: the row carries the factor T of Sec. 4.8, so u_g -> 0 satisfies it.)"""
    cfg, cases = cold_cases(count=8, seed=11)
    p = O.make_params(cfg)
    n = 1.0 / (cfg["gam"] - 1.0)
    for U, Ps, P in cases:
        s_true = n * math.log((cfg["gam"] - 1.0) * P[UU]) - (n + 1.0) * math.log(P[RHO])
        _, info = O.implicit_zone(p, X, U, Ps, 0.1, Sstar=U[RHO] * s_true)
        assert info.entropy == 1 and info.cold == 0 and info.e_T <= 1e-7
        _, info = O.implicit_zone(p, X, U, Ps, 0.1, Sstar=math.nan)
        assert info.entropy == 0 and info.cold == 1
        V = U.copy()
        V[UR1:UR3 + 1] *= 2.0 / np.linalg.norm(V[UR1:UR3 + 1]) * (-V[ER])
        _, info = O.implicit_zone(p, X, V, Ps, 0.1)
        assert info.cold == 0 and info.method == O.BACKUP
