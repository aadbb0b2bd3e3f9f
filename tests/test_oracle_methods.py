"""The oracle's three Newton formulations of the implicit four-force system
(Sec. 4.8): PMHD iterates the gas primitives, URAD the radiation conserved
quantities R^t_nu, PRAD the radiation primitives (Ebar, u~_rad); each
recovers the rest from total energy-momentum conservation.  They solve the
same equations (Eq. source3), so wherever two of them converge (e_T < 1e-9)
they must reach the same root.  On seeded random states (gas Lorentz factors
up to 5, radiation frames up to 3, Minkowski and Kerr-Schild) the URAD and
PRAD roots agree with the PMHD root to 1e-9 in the median and 1e-5 at worst
(an e_T of 1e-9 bounds the residual, not each primitive, where the system is
ill-conditioned), and each method converges on most states.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W


@pytest.mark.parametrize("metric", [0, 1])
def test_three_methods_reach_the_same_root(metric):
    cfg, x, P = W.random_states(120, seed=201 + metric, metric=metric, gamma_max=5.0, gamma_rad_max=3.0)
    cfg.update(kappa_abs0=3.0, kappa_es0=1.0)
    p = O.make_params(cfg)
    g = W.rng(5)
    h = 10 ** g.uniform(-3, 0, len(x))
    conv = np.zeros(3, dtype=int)
    diffs = {1: [], 2: []}
    for n in range(len(x)):
        U, _ = O.prim_to_cons(p, x[n], P[n])
        Ps = P[n].copy()
        Ps[W.UU] *= 1.0 + 0.3 * g.uniform(-1, 1)
        Ps[W.ER] *= 1.0 + 0.3 * g.uniform(-1, 1)
        res = [O.method_zone(p, x[n], U, Ps, h[n], m) for m in range(3)]
        for m in range(3):
            conv[m] += res[m][1] < 1e-9
        if res[0][1] < 1e-10:
            for m in (1, 2):
                if res[m][1] < 1e-9:
                    a, b = res[0][0], res[m][0]
                    idx = [W.RHO, W.UU, W.ER]
                    diffs[m].append(np.max(np.abs(a[idx] - b[idx]) / np.abs(a[idx])))
    print("converged PMHD/URAD/PRAD:", conv, "of", len(x),
          {m: (np.median(d), np.max(d)) for m, d in diffs.items()})
    assert conv.min() > 0.6 * len(x)
    for m in (1, 2):
        assert len(diffs[m]) > 0.5 * len(x)
        assert np.median(diffs[m]) < 1e-9 and np.max(diffs[m]) < 1e-5
