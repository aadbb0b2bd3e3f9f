"""Radiative shock tubes (Sec. 5, HD radiative shocks; Table t.radtube in
tests/golden/radiative_shocks.json) on the CUDA step.

Parity: 800 zones over [-20, 20] with zero-gradient ends that let the inflow
in (HARMRAD_BC_COPY), 20 steps of CUDA and oracle from the printed left/right
states; tests 1 (non-relativistic, radiation 1e-4 of the gas energy: many
URAD zones), 3b (upstream u^x = 10, optically thick) and 4a (radiation
pressure dominated).

Stationary shocks: tests 2, 3b and 4b run on the GPU to t = 300 (the time
the paper evolves them to).  The printed states are the asymptotic states of
a shock at rest, so the run must settle with the far states unchanged and the
total flux of rest mass, energy and momentum the same in every zone (a steady
state of a conservative scheme); the tolerance is the jump-condition rounding
of the printed states plus the smoothing of the shock by the scheme.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.parity_metrics import zone_errors
from tests.test_oracle_shocks import total_flux

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "radiative_shocks.json")))


def zone_total_flux(cfg, P12):
    """Total x-fluxes (rest mass, energy incl. rest mass, x-momentum) of the
    primitives of one zone, from the oracle's flux function."""
    F, _ = O.flux(O.make_params(cfg), [0.5, 0.5, 0.5], 1, P12)
    return np.array([F[0], F[1] + F[8], F[2] + F[9]])


def state(name):
    st = dict(GOLD["tests"][name])
    st["gam"] = float(Fraction(st["gam"]))
    return st


@pytest.mark.parametrize("name", ["1", "3b", "4a"])
def test_shock_tube_matches_oracle(name):
    cfg, P = W.shock_tube(state(name))
    g = H.Grid(cfg)
    g.set_prims(P)
    o = O.Oracle(cfg)
    o.set_prims(P)
    urad = np.zeros(P.shape[1:], dtype=bool)
    for _ in range(20):
        # the CFL dt follows the states, which agree to the Newton tolerance
        d = o.cfl_dt()
        assert g.cfl_dt() == pytest.approx(d, rel=1e-8)
        o.step(d)
        g.step(d)
        urad |= (o.status() != 0) | (g.status() != 0)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    ok = ~urad
    print("test %s: PMHD zones %.4e (%d), URAD/back-up zones %.4e (%d)"
          % (name, e[:, ok].max() if ok.any() else 0, ok.sum(), e[:, urad].max() if urad.any() else 0, urad.sum()))
    assert e[:, ok].max() < 1e-8, e[:, ok].reshape(12, -1).max(axis=1)
    if urad.any():
        assert e[:, urad].max() < 1e-6


@pytest.mark.parametrize("name", ["2", "3b", "4b"])
def test_shock_stands_still(name):
    st = state(name)
    cfg, P = W.shock_tube(st)
    g = H.Grid(cfg)
    g.set_prims(P)
    t = 0.0
    while t < 300.0:
        dt = min(g.cfl_dt(), 300.0 - t)
        g.step(dt)
        t += dt
    Q = g.get_prims()
    assert np.isfinite(Q).all()
    sig = float(st["sigma"])
    F = np.array([zone_total_flux(cfg, Q[:, 0, 0, i]) for i in range(Q.shape[-1])])
    FL = total_flux(st["gam"], sig, [float(v) for v in st["L"]])
    dev = np.abs(F - FL).max(axis=0) / np.abs(FL)
    far = np.abs(Q[:, 0, 0, :40] - P[:, 0, 0, :40]).max(axis=1)
    print("test %s: flux deviation %s; far-left drift rho %.2e ug %.2e ux %.2e E %.2e"
          % (name, dev, far[0], far[1], far[2], far[8]))
    assert dev.max() < 2e-2
