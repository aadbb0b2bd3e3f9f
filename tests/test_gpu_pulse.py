"""The optically thick radiation pulse (Sec. 5, planar pulse) on the CUDA step:
radiation 25 orders below the gas energy, so every zone is extremely
sub-dominant (Sec. 4.10) and the update kernel hands it to URAD in the retry
kernel.  Against the oracle over 20 steps (radiation energy to 1e-6 of the
peak, radiation velocity to 1e-6 of its largest value: URAD stops at
e_T < 1e-9 on both sides), and against the closed-form diffusion solution at
the times of the paper's figure as the oracle is (tests/test_oracle_pulse.py);
and the optically thin 3D pulse against the paper's printed peaks and the
oracle.
"""
import numpy as np

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.test_oracle_pulse import TIMES

import pytest

pytestmark = pytest.mark.gpu


def test_thick_pulse_matches_oracle():
    cfg, P = W.thick_pulse()
    g = H.Grid(cfg)
    g.set_prims(P)
    o = O.Oracle(cfg)
    o.set_prims(P)
    for _ in range(20):
        # the CFL step follows states that agree to the URAD tolerance
        d = o.cfl_dt()
        assert g.cfl_dt() == pytest.approx(d, rel=1e-7)
        o.step(d)
        g.step(d)
        assert np.all(g.status() == H.ZONE_URAD)
        assert np.all(o.status() == O.OK_URAD)
    A, R = g.get_prims(), o.get_prims()
    eE = np.abs(A[W.ER] - R[W.ER]).max() / R[W.ER].max()
    eu = np.abs(A[W.UR1] - R[W.UR1]).max() / np.abs(R[W.UR1]).max()
    eg = np.abs(A[W.UU] - R[W.UU]).max() / R[W.UU].max()
    print("Ebar %.2e, u~_rad %.2e, u_g %.2e" % (eE, eu, eg))
    assert eE < 1e-6 and eu < 1e-6 and eg < 1e-12


def test_thick_pulse_follows_diffusion_on_gpu():
    cfg, P = W.thick_pulse()
    g = H.Grid(cfg)
    g.set_prims(P)
    x = cfg["x0"][0] + (np.arange(cfg["n"][0]) + 0.5) * cfg["dx"][0]
    t = 0.0
    for T in TIMES:
        while t < T - 1e-9:
            dt = min(g.cfl_dt(), T - t)
            g.step(dt)
            t += dt
        E = g.get_prims()[W.ER].ravel()
        Ex = W.thick_pulse_exact(x, t)
        err = np.abs(E - Ex).max() / (Ex.max() - Ex.min())
        print("t = %.2f: err/peak %.3e" % (t, err))
        assert err < 3e-2


def test_thin_pulse_matches_paper_and_oracle():
    """The optically thin 3D pulse at 50^3 (Sec. 5; the paper's contour
    ranges in tests/golden/thin_pulse.json): the CUDA step's peak -R^t_t
    after free streaming to t = 15.21 and 35.01 is the paper's within 3 % and
    7 % (the oracle's is 2.1 % and 5.4 % below), and at t = 15.21 it matches
    the oracle zone by zone (URAD everywhere: 1e-6 of the peak)."""
    import os
    from tests.test_oracle_pulse import THIN, lab_energy
    os.environ["ORACLE_THREADS"] = str(os.cpu_count() or 1)
    cfg, P = W.thin_pulse()
    g = H.Grid(cfg)
    g.set_prims(P)
    o = O.Oracle(cfg)
    o.set_prims(P)
    t = 0.0
    c1, c2 = THIN["contours"][1], THIN["contours"][2]
    while t < c1["t"] - 1e-9:
        # radiation velocities near the gamma_rad cap at the front make the
        # signal speeds sensitive to the URAD tolerance: the CFL steps agree to 1e-5
        dt = min(o.cfl_dt(), c1["t"] - t)
        assert g.cfl_dt() == pytest.approx(o.cfl_dt(), rel=1e-5)
        o.step(dt)
        g.step(dt)
        t += dt
    Eg, Eo = lab_energy(g.get_prims()), lab_energy(o.get_prims())
    d = np.abs(Eg - Eo).max() / Eo.max()
    print("t = %.2f: GPU peak %.4e, oracle %.4e, paper %.4e, max difference %.2e of the peak"
          % (t, Eg.max(), Eo.max(), c1["max"], d))
    assert d < 1e-6
    assert abs(Eg.max() / c1["max"] - 1.0) < 0.03
    while t < c2["t"] - 1e-9:
        dt = min(g.cfl_dt(), c2["t"] - t)
        g.step(dt)
        t += dt
    Eg = lab_energy(g.get_prims())
    print("t = %.2f: GPU peak %.4e, paper %.4e" % (t, Eg.max(), c2["max"]))
    assert abs(Eg.max() / c2["max"] - 1.0) < 0.07
