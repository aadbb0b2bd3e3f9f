"""Batched contexts (several independent grids advanced by the same kernel
launches) and the per-zone absorption field (opacity mode 2).

- a batch steps every box exactly as a single-grid context steps that box
  (bit for bit, per-box CFL time steps included);
- small batches against the FP64 oracle box by box, 1 and 5 steps;
- the full 48-box workload (edges log-uniform in 32..128, optical depth per
  cell log-uniform over 1e-4..1e6): batch equals single grids on a sample of
  boxes, the smallest box against the oracle, heavy-tailed Newton counts.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.parity_metrics import zone_errors

pytestmark = pytest.mark.gpu


def single(cfg, P, K):
    g = H.Grid(cfg)
    g.set_prims(P)
    g.set_opacity_field(K)
    return g


def test_opacity_field_needs_field_mode():
    cfg, P = W.minkowski_box((8, 8, 8), seed=2)
    g = H.Grid(cfg)
    with pytest.raises(H.HarmradError):
        g.set_opacity_field(np.ones(P.shape[1:]))


def test_opacity_field_rejects_negative():
    cfgs, Ps, Ks = W.box_batch(count=1, edge=(8, 8), seed=1)
    g = H.Grid(cfgs[0])
    K = Ks[0].copy()
    K[0, 0, 0] = -1.0
    with pytest.raises(H.HarmradError):
        g.set_opacity_field(K)


def test_batch_rejects_mixed_physics():
    cfgs, _, _ = W.box_batch(count=2, edge=(8, 12), seed=1)
    cfgs[1] = dict(cfgs[1], gam=4.0 / 3.0)
    with pytest.raises(H.HarmradError):
        H.Batch(cfgs)


def test_batch_equals_single_grids():
    """Five boxes of 4..20 zones per edge, two CFL steps: every box of the
    batch ends bit for bit where its own single-grid context ends, with the
    same per-zone solver outcome and Newton counts."""
    cfgs, Ps, Ks = W.box_batch(count=5, edge=(4, 20), seed=99)
    bt = H.Batch(cfgs)
    bt.set_prims(Ps)
    bt.set_opacity_field(Ks)
    dts = []
    for c, P, K in zip(cfgs, Ps, Ks):
        dts.append(single(c, P, K).cfl_dt())
    assert bt.cfl_dt() == min(dts)
    for _ in range(2):
        bt.step(0.0)
    out, st, it = bt.get_prims(), bt.status(), bt.iters()
    for b, (c, P, K) in enumerate(zip(cfgs, Ps, Ks)):
        g = single(c, P, K)
        for _ in range(2):
            g.step(0.0)
        assert np.array_equal(g.get_prims(), out[b]), b
        assert np.array_equal(g.status(), st[b]), b
        assert np.array_equal(g.iters(), it[b]), b


@pytest.mark.parametrize("steps,tol", [(1, 1e-10), (5, 1e-8)])
def test_batch_against_oracle(steps, tol):
    """Three boxes (6..10 zones per edge) with the per-zone absorption field,
    each box on its own CFL step, against the oracle run box by box."""
    cfgs, Ps, Ks = W.box_batch(count=3, edge=(6, 10), seed=4242)
    bt = H.Batch(cfgs)
    bt.set_prims(Ps)
    bt.set_opacity_field(Ks)
    orcs = []
    for c, P, K in zip(cfgs, Ps, Ks):
        o = O.Oracle(c)
        o.set_prims(P)
        o.set_opacity_field(K)
        orcs.append(o)
    for _ in range(steps):
        bt.step(0.0)
        for o in orcs:
            o.step(0.0)
    out = bt.get_prims()
    for b, (c, o) in enumerate(zip(cfgs, orcs)):
        R = o.get_prims()
        e = zone_errors(c, out[b], R)
        ok = e.max(0) <= tol
        print("box %d %s: worst %.2e, zones over %.0e: %d of %d" %
              (b, c["n"], e.max(), tol, (~ok).sum(), ok.size))
        assert ok.all(), (b, e.max())


@pytest.fixture(scope="module")
def batch48():
    return W.box_batch()


def test_full_batch_equals_single_grids(batch48):
    """The 48-box workload (19.5 M zones): one CFL step of the batch equals,
    bit for bit, the single-grid step of the smallest, the largest and two
    other boxes."""
    cfgs, Ps, Ks = batch48
    bt = H.Batch(cfgs)
    bt.set_prims(Ps)
    bt.set_opacity_field(Ks)
    bt.step(0.0)
    s = bt.stats()
    out = bt.get_prims(device=True)
    assert torch.isfinite(out).all()
    sizes = [int(np.prod(c["n"])) for c in cfgs]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 31})
    for b in pick:
        o, m = int(bt.offsets[b]), bt.sizes[b]
        A = out[12 * o:12 * (o + m)].reshape(bt.shapes[b])
        g = single(cfgs[b], Ps[b], Ks[b])
        g.step(0.0)
        assert torch.equal(g.get_prims(device=True), A), b
        del g
    print("batch48 one step:", s)


def test_full_batch_smallest_box_against_oracle(batch48):
    """The smallest of the 48 boxes, one CFL step inside the batch, against
    the oracle (1e-10 per zone), and the heavy tail of the Newton counts."""
    cfgs, Ps, Ks = batch48
    bt = H.Batch(cfgs)
    bt.set_prims(Ps)
    bt.set_opacity_field(Ks)
    bt.step(0.0)
    sizes = [int(np.prod(c["n"])) for c in cfgs]
    b = int(np.argmin(sizes))
    A = bt.get_prims()[b]
    its = np.concatenate([i.ravel() for i in bt.iters()])
    o = O.Oracle(cfgs[b])
    o.set_prims(Ps[b])
    o.set_opacity_field(Ks[b])
    o.step(0.0)
    e = zone_errors(cfgs[b], A, o.get_prims())
    q = np.quantile(its, [0.5, 0.9, 0.99, 0.999])
    print("box %s: worst %.2e; Newton iterations per zone-step median/p90/p99/p99.9/max:"
          % (cfgs[b]["n"], e.max()), q, its.max())
    assert (e.max(0) <= 1e-10).all()
    assert its.max() > 2 * q[0]
