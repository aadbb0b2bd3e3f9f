"""Pins of the oracle's IMEX time integrators (Sec. 4.1, Eqs. IMEX2, IMEX2B,
IMEX3) by their order of accuracy on a stiff relaxation problem.

A uniform, static box of gas and radiation out of equilibrium exchanges
energy through absorption only: du_g/dt = kappa (Ebar - a_rad T^4),
T = (gam - 1) u_g / rho0, with u_g + Ebar conserved.  Every flux difference
vanishes, so each scheme reduces to its implicit (diagonally implicit RK)
part.  The reference solution comes from scipy's 8th-order Dormand-Prince
integrator of that ODE (not from the oracle); the relaxation rate is about 5
per unit time, so the coarsest steps are stiff (rate x dt > 1).  The measured
orders must be those of the schemes: 2 for IMEX2 and IMEX2B, 3 for IMEX3.
The RK3 scheme with the same coefficients for both parts (the paper's runs)
is first order for the stiff part: its error ratio tends to 2.

A restatement of the same stages for the scalar ODE (coefficients from the
printed equations, root of each implicit stage by bracketing) reproduces the
oracle's result; the same restatement with one coefficient wrong loses the
order, so the order test tells a mistyped coefficient apart.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

GAM, RHO, UG0, E0, KAPPA, TEND = 5.0 / 3.0, 1.0, 1e-2, 3e-2, 1.0, 1.0
T0 = (GAM - 1.0) * UG0 / RHO
A_RAD = 1e-2 / T0 ** 4
NS = [8, 16, 32, 64, 128]


def box(integrator):
    cfg = W.base_params()
    cfg.update(n=[4, 1, 1], dx=[0.25, 1.0, 1.0], a_rad=A_RAD, kappa_abs0=KAPPA, kappa_es0=0.0,
               integrator=integrator, newton_tol=1e-14)
    P = np.zeros((W.NP, 1, 1, 4))
    P[W.RHO], P[W.UU], P[W.ER] = RHO, UG0, E0
    return cfg, P


def rate(ug, C):
    return KAPPA * RHO * ((C - ug) - A_RAD * ((GAM - 1.0) * ug / RHO) ** 4)


def reference():
    C = UG0 + E0
    s = solve_ivp(lambda t, y: [rate(y[0], C)], [0.0, TEND], [UG0], method="DOP853", rtol=2.3e-14,
                  atol=1e-18)
    return s.y[0, -1]


def oracle_run(integrator, N):
    cfg, P = box(integrator)
    o = O.Oracle(cfg)
    o.set_prims(P)
    for _ in range(N):
        o.step(TEND / N)
    Q = o.get_prims()
    assert np.all(Q[W.UU] == Q[W.UU, 0, 0, 0])
    return Q[W.UU, 0, 0, 0]


def orders(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


@pytest.fixture(scope="module")
def ref():
    return reference()


@pytest.mark.parametrize("integrator,order", [(W.IMEX2, 2), (W.IMEX2B, 2), (W.IMEX3, 3)])
def test_imex_order_on_stiff_relaxation(ref, integrator, order):
    errs = [abs(oracle_run(integrator, N) - ref) for N in NS]
    p = orders(errs)
    print(integrator, ["%.3e" % e for e in errs], ["%.2f" % x for x in p])
    assert abs(p[-1] - order) < 0.15 and abs(p[-2] - order) < 0.25, p


def test_rk3_same_coefficients_is_first_order_when_stiff(ref):
    errs = [abs(oracle_run(W.RK3, N) - ref) for N in NS]
    p = orders(errs)
    assert p[-1] < 1.3 and p[0] > p[-1], p
    e3 = abs(oracle_run(W.IMEX3, NS[-1]) - ref)
    assert e3 < 1e-3 * errs[-1]


# --- scalar restatement of the printed stages ------------------------------

def stages(integrator, wrong=False):
    """(an, ap, d, c[], g) per stage; F = 0 here, so d never contributes."""
    if integrator == W.IMEX2:
        ga = 1.0 - 1.0 / math.sqrt(2.0)
        return [(1, 0, 0, [], ga),
                ((3 * ga - 1) / ga, (1 - 2 * ga) / ga, 1, [], ga),
                (0.5, 0.5, 0.5, [ga, (1 - ga) / 2 + (0.01 if wrong else 0.0)], 0.0)]
    al, be, et = 0.24169426078821, 0.06042356519705, 0.12915286960590
    return [(1, 0, 0, [], al),
            (2, -1, 0, [], al),
            (1, 0, 1, [0, 1 - al], al),
            (0.75, 0.25, 0.25, [be, (-1 + al + 4 * et) / 4, (2 - 5 * al - 4 * (be + et)) / 4 + (0.01 if wrong else 0.0)], al),
            (1 / 3, 2 / 3, 2 / 3, [-2 * be / 3, (1 - 4 * et) / 6, (-1 + 4 * al + 4 * (be + et)) / 6, 4 * (1 - al) / 6], 0.0)]


def scalar_run(integrator, N, wrong=False):
    C = UG0 + E0
    dt = TEND / N
    ug = UG0
    for _ in range(N):
        un, prev, M = ug, ug, []
        for an, ap, _, c, g in stages(integrator, wrong):
            us = an * un + ap * prev + dt * sum(cj * mj for cj, mj in zip(c, M))
            if g > 0.0:
                h = g * dt
                u = brentq(lambda x: x - us - h * rate(x, C), 0.0, C, xtol=1e-17, rtol=1e-15)
                M.append((u - us) / h)
            else:
                u = us
            prev = u
        ug = prev
    return ug


@pytest.mark.parametrize("integrator", [W.IMEX2, W.IMEX3])
def test_scalar_restatement_matches_oracle(integrator):
    for N in (8, 32):
        a, b = scalar_run(integrator, N), oracle_run(integrator, N)
        assert abs(a - b) < 1e-11 * UG0, (N, a, b)


@pytest.mark.parametrize("integrator,order", [(W.IMEX2, 2), (W.IMEX3, 3)])
def test_wrong_coefficient_loses_the_order(ref, integrator, order):
    errs = [abs(scalar_run(integrator, N, wrong=True) - ref) for N in NS]
    p = orders(errs)
    assert abs(p[-1] - order) > 0.5, p
