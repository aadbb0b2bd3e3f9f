"""The CUDA step on the linear-wave eigenmodes the paper prints (Sec. 5,
Table t.waves): one period of each mode in a 1D periodic box of 128 zones;
the measured omega (wave speed and damping rate) against the printed one,
as the oracle does in test_oracle_waves.py."""
import pytest

from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.test_oracle_waves import CASES, GOLD, N, measure_omega, tolerance

pytestmark = pytest.mark.gpu


class GridStepper:
    def __init__(self, cfg, P):
        self.g = H.Grid(cfg)
        self.g.set_prims(P)

    def cfl(self):
        return self.g.cfl_dt()

    def step(self, dt):
        self.g.step(dt)

    def rho(self):
        return self.g.get_prims()[0]


@pytest.mark.parametrize("case", CASES)
def test_gpu_linear_wave_omega(case):
    # FP64 only: the eigenmodes have relative amplitude 1e-6, below what FP32
    # face states resolve against the background
    precision = H.PREC_FP64
    mode = GOLD["cases"][case]
    cfg, P = W.linear_wave(N, GOLD["background"], mode)
    cfg = dict(cfg, precision=precision)
    w_re, w_im = measure_omega(GridStepper(cfg, P), cfg, P, mode["omega"][0])
    e_re = abs(w_re / mode["omega"][0] - 1)
    e_im = abs(w_im / mode["omega"][1] - 1)
    print("%s precision %d: omega %.6f + %.6f i (paper %.6f + %.6f i): rel err %.1e, %.1e"
          % (case, precision, w_re, w_im, mode["omega"][0], mode["omega"][1], e_re, e_im))
    t_re, t_im = tolerance(case)
    assert e_re < t_re
    assert e_im < t_im
