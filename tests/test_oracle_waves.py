"""Pin of the oracle against the linear-wave eigenmodes the paper prints
(Sec. 5, Table t.waves; values in tests/golden/linear_waves.json).  The
printed eigenvalues are those of the linearised equations with absorption
opacity tau and no scattering (the text calls the opacity scattering; with
scattering alone, or with both, the eigenvalues differ in the second digit):
the oracle runs them that way.

Each case starts a 1D periodic box from one printed eigenvector and evolves
it for one period P = 2 pi / Re(omega); the complex amplitude of the density
mode then gives the measured omega = -i ln(A(P)/A(0)) / P, whose real part
(wave speed) and imaginary part (damping by radiation diffusion) must match
the printed omega.  This pins, against numbers from the paper, the coupling
of gas and radiation through scattering, radiation pressure and the M1
closure, the fast and slow magnetosonic structure, and the time stepping.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "linear_waves.json")))
N = 128
CASES = list(GOLD["cases"])


def tolerance(case):
    """Relative tolerances on (Re omega, Im omega) at 128 zones: 1e-4 and 2e-2;
    3e-3 and 2e-2 for panel (d), optically thick and radiation dominated,
    whose modes lose 60-78 % of their amplitude in one period, so that the
    measured phase carries the scheme's damping error too (the oracle's
    errors there are 2e-4 to 1.8e-3)."""
    return (3e-3, 2e-2) if case.startswith("d_") else (1e-4, 2e-2)


def measure_omega(stepper, cfg, P, omega_re):
    k = GOLD["background"]["k"]
    period = 2 * math.pi / omega_re
    dt0 = stepper.cfl()
    m = int(math.ceil(period / dt0))
    dt = period / m
    A0 = W.wave_amplitude(P[0], k)
    for _ in range(m):
        stepper.step(dt)
    A1 = W.wave_amplitude(stepper.rho(), k)
    ratio = A1 / A0
    phase = math.atan2(ratio.imag, ratio.real)
    return (2 * math.pi + phase) / period, -math.log(abs(ratio)) / period


class OracleStepper:
    def __init__(self, cfg, P):
        self.o = O.Oracle(cfg)
        self.o.set_prims(P)

    def cfl(self):
        return self.o.cfl_dt()

    def step(self, dt):
        self.o.step(dt)

    def rho(self):
        return self.o.get_prims()[0]


@pytest.mark.parametrize("case", CASES)
def test_oracle_linear_wave_omega(case):
    mode = GOLD["cases"][case]
    cfg, P = W.linear_wave(N, GOLD["background"], mode)
    w_re, w_im = measure_omega(OracleStepper(cfg, P), cfg, P, mode["omega"][0])
    e_re = abs(w_re / mode["omega"][0] - 1)
    e_im = abs(w_im / mode["omega"][1] - 1)
    print("%s: omega %.6f + %.6f i (paper %.6f + %.6f i): rel err %.1e, %.1e"
          % (case, w_re, w_im, mode["omega"][0], mode["omega"][1], e_re, e_im))
    t_re, t_im = tolerance(case)
    assert e_re < t_re
    assert e_im < t_im


@pytest.mark.parametrize("integrator", [W.IMEX2, W.IMEX2B, W.IMEX3])
@pytest.mark.parametrize("case", ["a_sound", "a_fast", "a_slow", "c_sound", "b_sound"])
def test_oracle_linear_wave_omega_imex(case, integrator):
    """The printed eigenvalues with the IMEX integrators of Sec. 4.1 in place
    of RK3: the same tolerances (at 128 zones the spatial error dominates)."""
    mode = GOLD["cases"][case]
    cfg, P = W.linear_wave(N, GOLD["background"], mode)
    cfg["integrator"] = integrator
    w_re, w_im = measure_omega(OracleStepper(cfg, P), cfg, P, mode["omega"][0])
    assert abs(w_re / mode["omega"][0] - 1) < 1e-4
    assert abs(w_im / mode["omega"][1] - 1) < 2e-2


@pytest.mark.parametrize("case,order", [("a_sound", 2.0), ("c_fast", 2.0), ("d_sound", 0.9)])
def test_oracle_spatial_convergence(case, order):
    """Error of the measured omega against the printed one at 32, 64 and 128
    zones: the optically thin modes converge at least at second order (PPM on
    a smooth wave), the optically thick radiation-dominated mode at first
    order (the paper: the stiff terms are first order in space for optically
    thick waves, and its convergence figure shows both slopes)."""
    mode = GOLD["cases"][case]
    errs = []
    for n in (32, 64, 128):
        cfg, P = W.linear_wave(n, GOLD["background"], mode)
        w_re, w_im = measure_omega(OracleStepper(cfg, P), cfg, P, mode["omega"][0])
        errs.append(abs(complex(w_re, w_im) - complex(*mode["omega"])) / abs(complex(*mode["omega"])))
    p = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print(case, errs, p)
    assert np.all(p > order), p
