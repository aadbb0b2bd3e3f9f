"""The optically thick radiation pulse (Sec. 5, planar pulse) on the CUDA step:
radiation 25 orders below the gas energy, so every zone is extremely
sub-dominant (Sec. 4.10) and the update kernel hands it to URAD in the retry
kernel.  Against the oracle over 20 steps (radiation energy to 1e-6 of the
peak, radiation velocity to 1e-6 of its largest value: URAD stops at
e_T < 1e-9 on both sides), and against the closed-form diffusion solution at
the times of the paper's figure as the oracle is (tests/test_oracle_pulse.py).
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
