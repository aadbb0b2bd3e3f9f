"""The oracle's Newton formulations of the implicit four-force system
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


@pytest.mark.parametrize("metric", [0, 1])
def test_staged_pmhd(metric):
    """The staged PMHD of Sec. 4.10 (one momentum-only step damped by 1/2,
    energy-only steps, the first damped by 1/2, then the full 4D Newton, its
    first step damped by 1/4, two-sided differences) solves the same
    equations: where it and the plain PMHD converge they reach the same root
    (1e-9 median, 1e-5 worst, as above).  Its damping is what it is for: from
    a guess with u_g a thousand times too large and the velocity reversed it
    converges on more states than the undamped plain PMHD, and from the
    ordinary guesses on at least as many."""
    cfg, x, P = W.random_states(120, seed=201 + metric, metric=metric, gamma_max=5.0, gamma_rad_max=3.0)
    cfg.update(kappa_abs0=3.0, kappa_es0=1.0)
    p = O.make_params(cfg)
    g = W.rng(5)
    h = 10 ** g.uniform(-3, 0, len(x))
    conv, bad, diffs = np.zeros(2, dtype=int), np.zeros(2, dtype=int), []
    for n in range(len(x)):
        U, _ = O.prim_to_cons(p, x[n], P[n])
        Ps = P[n].copy()
        Ps[W.UU] *= 1.0 + 0.3 * g.uniform(-1, 1)
        Ps[W.ER] *= 1.0 + 0.3 * g.uniform(-1, 1)
        r0, r3 = O.method_zone(p, x[n], U, Ps, h[n], 0), O.method_zone(p, x[n], U, Ps, h[n], 3)
        conv += [r0[1] < 1e-9, r3[1] < 1e-9]
        if r0[1] < 1e-10 and r3[1] < 1e-9:
            idx = [W.RHO, W.UU, W.ER]
            diffs.append(np.max(np.abs(r0[0][idx] - r3[0][idx]) / np.abs(r0[0][idx])))
        Pb = Ps.copy()
        Pb[W.UU] *= 1e3
        Pb[W.U1:W.U3 + 1] *= -1.0
        bad += [O.method_zone(p, x[n], U, Pb, h[n], m)[1] < 1e-9 for m in (0, 3)]
    print("converged plain/staged:", conv, "from the bad guess:", bad,
          "root difference median %.1e max %.1e" % (np.median(diffs), np.max(diffs)))
    assert conv[1] >= conv[0] and bad[1] > bad[0]
    assert len(diffs) > 0.5 * len(x) and np.median(diffs) < 1e-9 and np.max(diffs) < 1e-5


@pytest.mark.parametrize("metric", [0, 1])
def test_staged_radiation_methods(metric):
    """The staged URAD and PRAD of Sec. 4.10 (the staged PMHD's stages on the
    radiation unknowns, one-sided differences, 40 x 6 gas inversions) solve
    the same equations as the plain methods: where both converge they reach
    the same root (1e-9 median, 1e-5 worst), and they converge on most of
    the states."""
    cfg, x, P = W.random_states(120, seed=201 + metric, metric=metric, gamma_max=5.0, gamma_rad_max=3.0)
    cfg.update(kappa_abs0=3.0, kappa_es0=1.0)
    p = O.make_params(cfg)
    g = W.rng(5)
    h = 10 ** g.uniform(-3, 0, len(x))
    conv = np.zeros(6, dtype=int)
    diffs = {4: [], 5: []}
    for n in range(len(x)):
        U, _ = O.prim_to_cons(p, x[n], P[n])
        Ps = P[n].copy()
        Ps[W.UU] *= 1.0 + 0.3 * g.uniform(-1, 1)
        Ps[W.ER] *= 1.0 + 0.3 * g.uniform(-1, 1)
        res = {m: O.method_zone(p, x[n], U, Ps, h[n], m) for m in (1, 2, 4, 5)}
        for m in res:
            conv[m] += res[m][1] < 1e-9
        for m, base in ((4, 1), (5, 2)):
            if res[base][1] < 1e-9 and res[m][1] < 1e-9:
                idx = [W.RHO, W.UU, W.ER]
                diffs[m].append(np.max(np.abs(res[m][0][idx] - res[base][0][idx]) / np.abs(res[base][0][idx])))
    print("converged URAD/PRAD plain %d/%d, staged %d/%d;" % (conv[1], conv[2], conv[4], conv[5]),
          {m: (np.median(d), np.max(d)) for m, d in diffs.items()})
    for m in (4, 5):
        assert conv[m] > 0.5 * len(x)
        assert np.median(diffs[m]) < 1e-9 and np.max(diffs[m]) < 1e-5
