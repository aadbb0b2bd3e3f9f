"""Pins of the oracle against the radiative shock tubes the paper prints
(Sec. 5, HD radiative shocks; Table t.radtube in
tests/golden/radiative_shocks.json).

Tests 1-4b list the two asymptotic states of a shock at rest on the grid, in
LTE (fluid-frame radiation energy a_rad T^4 with T = p_g / rho0, a_rad =
4 sigma_rad) and with the radiation moving with the gas.  A stationary shock
carries the same total flux of rest mass, energy and x-momentum on both sides,
so the oracle's flux function (gas stress-energy plus the M1 radiation tensor,
Eq. 751 conserved/flux set) evaluated at the printed left and right states
must agree within what the table's rounding allows: each printed value is
uncertain by half a unit of its last digit, and the bound is the linear
propagation of those uncertainties through the same flux function.  A dropped
or mis-signed pressure, radiation-pressure or Lorentz-factor term breaks the
jump condition by far more than the rounding for at least one of the tests
(the radiation-dominated 4a/4b and the ultra-relativistic 3a/3b especially).
Test 5 (two colliding flows) has no stationary state and must show a jump.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "radiative_shocks.json")))
STATIONARY = ["1", "2", "3a", "3b", "4a", "4b"]
X = [0.5, 0.5, 0.5]


def half_ulp(s):
    """Half a unit of the last printed digit of the decimal string s."""
    mant, _, exp = s.lower().partition("e")
    dec = len(mant.split(".")[1]) if "." in mant else 0
    return 0.5 * 10.0 ** (int(exp or 0) - dec)


def case(name):
    t = GOLD["tests"][name]
    gam = float(Fraction(t["gam"]))
    return gam, t


def total_flux(gam, sigma, state):
    """Total x-fluxes (rest mass, energy incl. rest mass, x-momentum) of an
    LTE state with comoving radiation, from the oracle's flux function."""
    rho, pg, ux, E = state
    cfg = W.base_params()
    cfg.update(gam=gam, a_rad=4.0 * sigma)
    p = O.make_params(cfg)
    P = np.zeros(W.NP)
    P[W.RHO], P[W.UU], P[W.U1], P[W.ER], P[W.UR1] = rho, pg / (gam - 1.0), ux, E, ux
    F, _ = O.flux(p, X, 1, P)
    return np.array([F[0], F[1] + F[8], F[2] + F[9]])


def jump_and_bound(name):
    gam, t = case(name)
    sig = float(t["sigma"])
    vals = [float(v) for v in t["L"]] + [float(v) for v in t["R"]]
    dv = [half_ulp(v) for v in t["L"]] + [half_ulp(v) for v in t["R"]]

    def jump(v):
        return total_flux(gam, sig, v[:4]) - total_flux(gam, sig, v[4:])

    j = jump(vals)
    bound = np.zeros(3)
    for i in range(8):
        h = 1e-4 * dv[i]
        vp = list(vals)
        vm = list(vals)
        vp[i] += h
        vm[i] -= h
        bound += np.abs((jump(vp) - jump(vm)) / (2 * h)) * dv[i]
    return j, bound, total_flux(gam, sig, vals[:4])


@pytest.mark.parametrize("name", STATIONARY)
def test_jump_conditions_hold_within_rounding(name):
    j, bound, FL = jump_and_bound(name)
    assert np.all(np.abs(j) <= bound + 1e-14 * np.abs(FL)), (name, j, bound)


def test_colliding_flows_are_not_stationary():
    j, bound, FL = jump_and_bound("5")
    assert np.any(np.abs(j) > bound), (j, bound)


@pytest.mark.parametrize("name", STATIONARY)
def test_states_are_in_lte(name):
    """The printed Ehat equals 4 sigma (p_g / rho0)^4 within rounding: the
    table's a_rad = 4 sigma_rad and gas temperature p_g / rho0 are the ones
    the workload uses."""
    gam, t = case(name)
    sig = float(t["sigma"])
    for side in ("L", "R"):
        rho, pg, _, E = (float(v) for v in t[side])
        drho, dpg, _, dE = (half_ulp(v) for v in t[side])
        model = 4.0 * sig * (pg / rho) ** 4
        rel = 4.0 * (dpg / pg + drho / rho) + half_ulp(t["sigma"]) / sig + dE / E
        assert abs(E / model - 1.0) <= rel, (name, side, E, model)


@pytest.mark.parametrize("mistake", ["none", "no_rad_pressure", "no_gas_pressure", "newtonian"])
def test_plausible_mistakes_break_a_jump_condition(mistake):
    """Restated fluxes with one term wrong (planted here, not in the oracle)
    violate the jump condition beyond rounding for some printed test: the pin
    can tell them apart.  Without a planted mistake the restatement equals the
    oracle's flux."""
    broken = False
    for name in STATIONARY:
        gam, t = case(name)
        sig = float(t["sigma"])
        j, bound, _ = jump_and_bound(name)

        def planted(state):
            rho, pg, ux, E = state
            ug = pg / (gam - 1.0)
            ut = 1.0 if mistake == "newtonian" else np.sqrt(1.0 + ux * ux)
            w = rho + ug + pg
            prad = 0.0 if mistake == "no_rad_pressure" else E / 3.0
            pgas = 0.0 if mistake == "no_gas_pressure" else pg
            Ttx = -w * ut * ut * ux / ut + 0.0
            Txx = w * ux * ux + pgas
            Rtx = -(4.0 / 3.0) * E * ut * ux
            Rxx = (4.0 / 3.0) * E * ux * ux + prad
            return np.array([rho * ux, Ttx + rho * ux + Rtx, Txx + Rxx])

        L = [float(v) for v in t["L"]]
        R = [float(v) for v in t["R"]]
        if mistake == "none":
            for st in (L, R):
                ref = total_flux(gam, sig, st)
                assert np.allclose(planted(st), ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
        jp = planted(L) - planted(R)
        if np.any(np.abs(jp) > bound + 1e-14):
            broken = True
    assert broken == (mistake != "none"), mistake
