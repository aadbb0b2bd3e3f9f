"""Pins of the oracle on the optically thick radiation pulse (Sec. 5, planar
pulse in 1D Cartesian Minkowski) and of the sub-dominance test that selects
its implicit method (Sec. 4.10).

The pulse (radiation temperature T_a (1 + 100 exp(-x^2/w^2)), T_a = 10^6 K,
w = 5, 100 zones on [-50, 50], kappa_es = 10^3, no absorption, a_rad =
8.77e-12 in code units as the paper gives it) carries radiation 25 orders
below the gas energy: every zone is "extremely sub-dominant" and takes URAD.
In the diffusion limit the radiation energy obeys dE/dt = D d2E/dx2 with
D = 1/(3 kappa_tot); the initial profile is a sum of Gaussians whose
spreading is known in closed form (workloads.thick_pulse_exact), so the
oracle's solution at the times of the paper's figure (t = 2951.05, 9867.95,
29877.1) must follow it to the scheme's accuracy: within 3 % of the peak at
100 zones and closer at 200 (the paper: the central points diffuse slightly
faster at first).  The radiation energy is conserved (no absorption) and no
zone takes the back-up.  A wrong diffusion coefficient (the M1 pressure
E/3, the scattering coupling, the optical-depth limit of the wave speeds)
moves the profile by far more than 3 %.  The leading Gaussian's time offset
t0 = 3 kappa w^2 / 16 = 4687.5 is the paper's t0 (about 4800).

The optically thin 3D pulse (same T_a and a_rad, w = 5, 50^3 zones on
[-50, 50)^3, no opacity) is pinned to the contour ranges the paper prints for
its run (tests/golden/thin_pulse.json): the initial extremes of -R^t_t are
the workload's to the printed digits (they fix T_a, w, a_rad and the grid),
and the peak after free streaming to t = 15.21 must be the paper's 5.963e-34
within 3 % (the oracle gives 2.1 % below; the flattener and limiter details
the paper leaves out differ), with the radiation energy conserved.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

THIN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "thin_pulse.json")))

TIMES = [2951.05, 9867.95, 29877.1]
TINY = 10.0 * 2.220446049250313e-16


def radiation_energy(cfg, P, x):
    """Sum over zones of the conserved radiation energy -R^t_t."""
    p = O.make_params(cfg)
    return -sum(O.prim_to_cons(p, [0.0, xi, 0.5, 0.5], P[:, 0, 0, i])[0][W.ER] for i, xi in enumerate(x))


def run(n1, times):
    cfg, P = W.thick_pulse(n1=n1)
    o = O.Oracle(cfg)
    o.set_prims(P)
    x = cfg["x0"][0] + (np.arange(n1) + 0.5) * cfg["dx"][0]
    E0 = radiation_energy(cfg, P, x)
    out, t = [], 0.0
    for T in times:
        while t < T - 1e-9:
            dt = min(o.cfl_dt(), T - t)
            o.step(dt)
            t += dt
            st = o.status()
            assert np.all(st == O.OK_URAD), np.bincount(st.ravel(), minlength=3)
        Q = o.get_prims()
        E = Q[W.ER].ravel()
        Ex = W.thick_pulse_exact(x, t)
        bg = Ex.min()
        out.append((np.abs(E - Ex).max() / (Ex.max() - bg), radiation_energy(cfg, Q, x) / E0))
    return out


def test_thick_pulse_follows_diffusion():
    res = run(100, TIMES)
    print(["err/peak %.3e, energy %.12f" % r for r in res])
    for err, en in res:
        assert err < 3e-2
        assert abs(en - 1.0) < 1e-9


def test_thick_pulse_error_falls_with_resolution():
    (e100, _), = run(100, TIMES[:1])
    (e200, _), = run(200, TIMES[:1])
    assert e200 < 0.7 * e100, (e100, e200)


def test_leading_gaussian_offset_is_the_papers():
    w, kappa = 5.0, 1e3
    t0 = 3.0 * kappa * w * w / 16.0
    assert abs(t0 / 4800.0 - 1.0) < 0.03


def _zone(E_over_ug, moving=0.0):
    cfg = W.base_params()
    p = O.make_params(cfg)
    x = [0.0, 0.5, 0.5, 0.5]
    P = np.zeros(W.NP)
    P[W.RHO], P[W.UU] = 1.0, 1e-3
    P[W.ER] = E_over_ug * 1e-3
    P[W.UR1] = moving
    U, _ = O.prim_to_cons(p, x, P)
    return p, x, U, P


@pytest.mark.parametrize("ratio,expect", [(1e-16, True), (1e-14, False), (1e-3, False)])
def test_subdominance_threshold(ratio, expect):
    """Radiation at rest in gas at rest: U*'s energy rows are -Ebar and -u_g
    (rest mass removed), Ehat = Ebar; the test fires below 10 eps_m."""
    p, x, U, P = _zone(ratio)
    assert O.radiation_subdominant(p, x, U, P) == expect


def test_subdominance_uses_the_fluid_frame_energy():
    """A radiation frame moving at u~ = 10 relative to the gas has
    Ehat = Ebar (4/3 gamma^2 - 1/3) = 134 Ebar: Ebar = 1e-16 u_g is not
    sub-dominant in the fluid frame.  U* is given a large radiation energy so
    that only the fluid-frame test decides."""
    p, x, U, P = _zone(1e-16, moving=10.0)
    U = U.copy()
    U[W.ER] = -1e-3
    assert not O.radiation_subdominant(p, x, U, P)
    P2 = P.copy()
    P2[W.ER] = 1e-20
    assert O.radiation_subdominant(p, x, U, P2)


def test_unchanged_radiation_is_not_subdominant():
    """A radiation field of the size of the gas energy that the explicit
    update left unchanged (uniform radiation, perturbed gas: the stiff
    relaxation box) is not sub-dominant."""
    cfg, P = W.relax_box(n1=16)
    p = O.make_params(cfg)
    for i in range(16):
        x = [0.0, (i + 0.5) / 16, 0.5, 0.5]
        U, _ = O.prim_to_cons(p, x, P[:, 0, 0, i])
        assert not O.radiation_subdominant(p, x, U, P[:, 0, 0, i])


def lab_energy(P):
    """-R^t_t in Minkowski: Ebar (4/3 gamma^2 - 1/3) of the radiation frame."""
    g2 = 1.0 + P[W.UR1] ** 2 + P[W.UR2] ** 2 + P[W.UR3] ** 2
    return P[W.ER] * ((4.0 / 3.0) * g2 - 1.0 / 3.0)


def test_thin_pulse_initial_extremes_are_the_papers():
    cfg, P = W.thin_pulse()
    E = lab_energy(P)
    c0 = THIN["contours"][0]
    assert abs(E.max() / c0["max"] - 1.0) < 5e-4
    assert abs(E.min() / c0["min"] - 1.0) < 1e-3


def test_thin_pulse_peak_after_free_streaming():
    os.environ["ORACLE_THREADS"] = str(os.cpu_count() or 1)
    cfg, P = W.thin_pulse()
    o = O.Oracle(cfg)
    o.set_prims(P)
    t, T = 0.0, THIN["contours"][1]["t"]
    E0 = lab_energy(P).sum()
    while t < T - 1e-9:
        dt = min(o.cfl_dt(), T - t)
        o.step(dt)
        t += dt
        assert np.all(o.status() == O.OK_URAD)
    E = lab_energy(o.get_prims())
    print("t = %.2f: max -R^t_t %.4e (paper %.4e), energy %.12f"
          % (t, E.max(), THIN["contours"][1]["max"], E.sum() / E0))
    assert abs(E.max() / THIN["contours"][1]["max"] - 1.0) < 0.03
    assert abs(E.sum() / E0 - 1.0) < 1e-8
