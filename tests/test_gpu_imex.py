"""The IMEX integrators (Sec. 4.1, Eqs. IMEX2, IMEX2B, IMEX3) on the CUDA step,
against the oracle and against their orders of accuracy.

- the stiff relaxation box of tests/test_oracle_imex.py: the CUDA step has
  the scheme's order (2, 2, 3) against scipy's reference solution;
- the stiff 1D relaxation box (tau = 10 per zone), a 3D Minkowski box (MC,
  HLL) and the Kerr-Schild torus against the oracle, per zone 1e-10 after
  one step, 1e-8 after ten (zones that took URAD or the back-up on either
  side excluded and counted, as in the RK3 parity tests).  IMEX3's second
  bracket [2 U^n - U^0] is taken as [U^n - alpha dt M^0] (the same by its
  first stage), so that it does not subtract what the floors added to the
  first stage's solution in the torus atmosphere;
- a batch of boxes (optical depth per cell up to 1e6) equals its
  single-grid contexts bit for bit, and matches the oracle box by box after
  two IMEX2B steps (eight sub-steps) to 1e-6 per zone: URAD, whose Newton
  stops at e_T < 1e-9, solves up to 7 % of the zones, and its differences
  reach their neighbours through the fluxes of every later sub-step;
- the adjoint refuses an IMEX context.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.parity_metrics import zone_errors
from tests.test_oracle_imex import NS, TEND, box, orders, reference

pytestmark = pytest.mark.gpu

SCHEMES = [W.IMEX2, W.IMEX2B, W.IMEX3]


def run_pair(cfg, P, steps):
    g = H.Grid(cfg)
    g.set_prims(P)
    o = O.Oracle(cfg)
    o.set_prims(P)
    bad = np.zeros(P.shape[1:], dtype=bool)
    for _ in range(steps):
        d = o.cfl_dt()
        assert g.cfl_dt() == pytest.approx(d, rel=1e-10)
        o.step(d)
        g.step(d)
        bad |= (o.status() != 0) | (g.status() != 0)
    return g, o, bad


@pytest.mark.parametrize("integrator,order", [(W.IMEX2, 2), (W.IMEX2B, 2), (W.IMEX3, 3)])
def test_gpu_imex_order(integrator, order):
    ref = reference()
    errs = []
    for N in NS:
        cfg, P = box(integrator)
        g = H.Grid(cfg)
        g.set_prims(P)
        for _ in range(N):
            g.step(TEND / N)
        errs.append(abs(g.get_prims()[W.UU, 0, 0, 0] - ref))
    p = orders(errs)
    print(integrator, ["%.3e" % e for e in errs], ["%.2f" % x for x in p])
    assert abs(p[-1] - order) < 0.15 and abs(p[-2] - order) < 0.25, p


@pytest.mark.parametrize("integrator", SCHEMES)
def test_relax_box_matches_oracle(integrator):
    cfg, P = W.relax_box(n1=256)
    cfg["integrator"] = integrator
    g, o, bad = run_pair(cfg, P, 3)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    assert not bad.any()
    assert e.max() < 1e-10, e.reshape(12, -1).max(axis=1)


@pytest.mark.parametrize("integrator", SCHEMES)
def test_minkowski_box_matches_oracle(integrator):
    cfg, P = W.minkowski_box(n=(20, 12, 9), seed=8, recon=W.MC, flux=W.HLL)
    cfg["integrator"] = integrator
    g, o, bad = run_pair(cfg, P, 1)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    assert e[:, ~bad].max() < 1e-10, e[:, ~bad].reshape(12, -1).max(axis=1)


@pytest.mark.parametrize("integrator,steps,tol", [(W.IMEX2, 1, 1e-10), (W.IMEX2B, 1, 1e-10), (W.IMEX2B, 10, 1e-8),
                                                  (W.IMEX3, 1, 1e-10), (W.IMEX3, 10, 1e-8)])
def test_torus_matches_oracle(integrator, steps, tol):
    cfg, P = W.torus((64, 32, 16), seed=12345)
    cfg["integrator"] = integrator
    g, o, bad = run_pair(cfg, P, steps)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    ok = ~bad
    print("IMEX %d, %d steps: excluded zones (URAD/back-up) %d of %d, worst %.2e"
          % (integrator, steps, int(bad.sum()), bad.size, e[:, ok].max()))
    assert ok.mean() > 0.9
    assert e[:, ok].max() < tol, e[:, ok].reshape(12, -1).max(axis=1)


def test_batch_imex_equals_single_grids_and_oracle():
    cfgs, Ps, Ks = W.box_batch(count=3, edge=(6, 10), seed=4242)
    cfgs = [dict(c, integrator=W.IMEX2B) for c in cfgs]
    bt = H.Batch(cfgs)
    bt.set_prims(Ps)
    bt.set_opacity_field(Ks)
    for _ in range(2):
        bt.step(0.0)
    out = bt.get_prims()
    for b, (c, P, K) in enumerate(zip(cfgs, Ps, Ks)):
        g = H.Grid(c)
        g.set_prims(P)
        g.set_opacity_field(K)
        o = O.Oracle(c)
        o.set_prims(P)
        o.set_opacity_field(K)
        bad = np.zeros(P.shape[1:], dtype=bool)
        for _ in range(2):
            g.step(0.0)
            o.step(0.0)
            bad |= (g.status() != 0) | (o.status() != 0)
        assert np.array_equal(g.get_prims(), out[b]), b
        e = zone_errors(c, out[b], o.get_prims())
        print("box %d: URAD/back-up zones %d of %d, worst PMHD zone %.2e, worst URAD zone %.2e"
              % (b, bad.sum(), bad.size, e[:, ~bad].max(), e[:, bad].max() if bad.any() else 0.0))
        assert e.max() < 1e-6, (b, e.max())


def test_adjoint_rejects_imex():
    cfg, P = W.minkowski_box((8, 8, 8), seed=5)
    cfg["integrator"] = W.IMEX3
    g = H.Grid(cfg)
    g.set_prims(P)
    with pytest.raises(H.HarmradError):
        g.adjoint_enable(True)
