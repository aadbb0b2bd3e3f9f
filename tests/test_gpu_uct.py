"""The staggered magnetic field with the 4-state upwind EMF (HARMRAD_EMF_UCT;
Sec. 4.2 steps viii-x) on the CUDA step, against the oracle:

- periodic Minkowski boxes (PPM + LAXF, MC + HLL) with a random field from a
  vector potential: primitives per zone within 1e-10 after one step, and the
  face fields within 1e-10 of the field scale;
- the Kerr-Schild torus with its potential's face field: 1e-10 after one step,
  1e-8 after ten (zones that took URAD or the back-up on either side excluded,
  as in the flux-CT parity tests), faces alike; one IMEX2 and one IMEX3 step
  at 1e-10;
- the face divergence keeps its initial value to round-off over 20 steps of
  the torus on the GPU;
- a batch of boxes initialised from cell-centred fields equals its single-grid
  contexts bit for bit;
- split precision tracks FP64 on the torus;
- the two field transports (flux-CT and the staggered field) compared on the
  torus after 20 steps: reported, with the total radial magnetic stress
  within 10 %;
- the adjoint refuses a staggered context.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from paper_1312_6127_gb300 import workloads as W
from tests.parity_metrics import zone_errors
from tests.test_oracle_uct import curl_faces, face_div

pytestmark = pytest.mark.gpu


def pair(cfg, P, Bf):
    g = H.Grid(cfg)
    g.set_prims(P)
    o = O.Oracle(cfg)
    o.set_prims(P)
    if Bf is not None:
        g.set_face_fields(Bf)
        o.set_face_fields(Bf)
    return g, o


def face_error(bg, bo):
    scale = max(np.abs(b).max() for b in bo)
    return max(np.abs(bg[i] - bo[i]).max() for i in range(3)) / scale


def box_case(recon, flux):
    cfg, P = W.minkowski_box((20, 12, 9), seed=8, recon=recon, flux=flux)
    cfg["emf"] = H.EMF_UCT
    g = W.rng(77)
    A = [0.02 * g.standard_normal((9, 12, 20)) for _ in range(3)]
    return cfg, P, curl_faces(A, cfg["dx"])


@pytest.mark.parametrize("recon,flux", [(W.PPM, W.LAXF), (W.MC, W.HLL)])
def test_box_matches_oracle(recon, flux):
    cfg, P, Bf = box_case(recon, flux)
    g, o = pair(cfg, P, Bf)
    assert np.allclose(g.get_prims()[5:8], o.get_prims()[5:8], rtol=1e-13, atol=1e-15)
    d = o.cfl_dt()
    assert g.cfl_dt() == pytest.approx(d, rel=1e-12)
    o.step(d)
    g.step(d)
    bad = (o.status() != 0) | (g.status() != 0)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    ef = face_error(g.get_face_fields(), o.get_face_fields())
    print("UCT box recon %d flux %d: worst zone %.2e, faces %.2e" % (recon, flux, e[:, ~bad].max(), ef))
    assert e[:, ~bad].max() < 1e-10 and ef < 1e-10


@pytest.mark.parametrize("steps,tol", [(1, 1e-10), (10, 1e-8)])
def test_torus_matches_oracle(steps, tol):
    cfg, P, Bf = W.torus((64, 32, 16), seed=12345, faces=True)
    cfg["emf"] = H.EMF_UCT
    g, o = pair(cfg, P, Bf)
    bad = np.zeros(P.shape[1:], dtype=bool)
    for _ in range(steps):
        d = o.cfl_dt()
        assert g.cfl_dt() == pytest.approx(d, rel=1e-10)
        o.step(d)
        g.step(d)
        bad |= (o.status() != 0) | (g.status() != 0)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    ef = face_error(g.get_face_fields(), o.get_face_fields())
    print("UCT torus, %d steps: excluded zones %d of %d, worst zone %.2e, faces %.2e"
          % (steps, int(bad.sum()), bad.size, e[:, ~bad].max(), ef))
    assert (~bad).mean() > 0.9
    assert e[:, ~bad].max() < tol and ef < tol


@pytest.mark.parametrize("integrator", [W.IMEX2, W.IMEX3])
def test_torus_imex_matches_oracle(integrator):
    """The face fields take the IMEX brackets' combinations (Sec. 4.1): one
    IMEX step of the torus against the oracle, 1e-10 per zone and face."""
    cfg, P, Bf = W.torus((64, 32, 16), seed=12345, faces=True)
    cfg.update(emf=H.EMF_UCT, integrator=integrator)
    g, o = pair(cfg, P, Bf)
    d = o.cfl_dt()
    o.step(d)
    g.step(d)
    bad = (o.status() != 0) | (g.status() != 0)
    e = zone_errors(cfg, g.get_prims(), o.get_prims())
    ef = face_error(g.get_face_fields(), o.get_face_fields())
    print("UCT torus, IMEX %d, 1 step: excluded zones %d, worst zone %.2e, faces %.2e"
          % (integrator, int(bad.sum()), e[:, ~bad].max(), ef))
    assert (~bad).mean() > 0.9 and e[:, ~bad].max() < 1e-10 and ef < 1e-10


def test_face_divergence_on_gpu():
    cfg, P, Bf = W.torus((64, 32, 16), seed=12345, faces=True)
    cfg["emf"] = H.EMF_UCT
    g = H.Grid(cfg)
    g.set_prims(P)
    g.set_face_fields(Bf)
    b0 = g.get_face_fields()
    scale = max(np.abs(b).max() for b in b0) / min(cfg["dx"])
    d0 = face_div(b0, cfg["dx"])
    for _ in range(20):
        g.step(0.0)
    b = g.get_face_fields()
    drift = np.abs(face_div(b, cfg["dx"]) - d0).max()
    change = max(np.abs(b[i] - b0[i]).max() for i in range(3)) / max(np.abs(x).max() for x in b0)
    print("UCT torus, 20 steps: relative field change %.2e, divergence drift %.2e of scale %.2e"
          % (change, drift, scale))
    assert change > 1e-6 and drift < 1e-13 * scale


def test_batch_equals_single_grids():
    cfgs, Ps, Ks = W.box_batch(count=3, edge=(6, 10), seed=4242)
    cfgs = [dict(c, emf=H.EMF_UCT) for c in cfgs]
    for P in Ps:  # a field for the boxes (the batch workload has none)
        P[5] = 0.05 * np.sin(2 * np.pi * np.arange(P.shape[3]) / P.shape[3])[None, None, :]
        P[6] = 0.03
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
        for _ in range(2):
            g.step(0.0)
        assert np.array_equal(g.get_prims(), out[b]), b


def test_split_precision_tracks_fp64():
    cfg, P, Bf = W.torus((64, 32, 16), seed=12345, faces=True)
    cfg["emf"] = H.EMF_UCT
    outs = []
    for prec in (H.PREC_FP64, H.PREC_SPLIT):
        g = H.Grid(cfg, precision=prec)
        g.set_prims(P)
        g.set_face_fields(Bf)
        for _ in range(3):
            g.step(0.0)
        outs.append((g.get_prims(), g.get_face_fields()))
    e = zone_errors(cfg, outs[1][0], outs[0][0])
    ef = face_error(outs[1][1], outs[0][1])
    print("UCT split vs FP64 after 3 steps: median zone %.2e, p99 %.2e, faces %.2e"
          % (np.median(e.max(axis=0)), np.quantile(e.max(axis=0), 0.99), ef))
    assert np.all(np.isfinite(outs[1][0])) and np.quantile(e.max(axis=0), 0.99) < 1e-3 and ef < 1e-3


def test_flux_ct_and_uct_on_the_torus():
    """Both transports from the same potential: after 20 steps the cell-centred
    fields differ at the level of the schemes' truncation error; the magnetic
    part of sum over zones of sqrt(-g) T^1_1 (the radial magnetic stress)
    agrees within 10 %."""
    cfg, P, Bf = W.torus((64, 32, 16), seed=12345, faces=True)
    res = {}
    for emf in (H.EMF_FLUXCT, H.EMF_UCT):
        c = dict(cfg, emf=emf)
        g = H.Grid(c)
        g.set_prims(P)
        if emf == H.EMF_UCT:
            g.set_face_fields(Bf)
        for _ in range(20):
            g.step(0.0)
        res[emf] = g.get_prims()
    p = O.make_params(cfg)

    def mag_stress(Q):
        tot = 0.0
        n1, n2, n3 = cfg["n"]
        for j in range(n2):
            for i in range(n1):
                x = [0.0, cfg["x0"][0] + (i + 0.5) * cfg["dx"][0], (j + 0.5) * cfg["dx"][1], 0.5]
                gcov, gcon, gdet = O.metric(p, x)[:3]
                for k in range(n3):
                    T, _ = O.stress(p, x, Q[:, k, j, i])
                    Qb = Q[:, k, j, i].copy()
                    Qb[5:8] = 0.0
                    T0, _ = O.stress(p, x, Qb)
                    tot += gdet * (T - T0)[1, 1]
        return tot
    e_ct, e_uct = mag_stress(res[H.EMF_FLUXCT]), mag_stress(res[H.EMF_UCT])
    dB = np.abs(res[H.EMF_UCT][5:8] - res[H.EMF_FLUXCT][5:8]).sum() / np.abs(res[H.EMF_FLUXCT][5:8]).sum()
    print("torus 64x32x16, 20 steps: flux-CT vs staggered field, relative L1 difference of B %.2e; "
          "magnetic stress T^1_1 total %.4e vs %.4e" % (dB, e_ct, e_uct))
    assert abs(e_uct - e_ct) < 0.1 * abs(e_ct)


def test_adjoint_rejects_uct():
    cfg, P = W.minkowski_box((8, 8, 8), seed=5)
    cfg["emf"] = H.EMF_UCT
    g = H.Grid(cfg)
    g.set_prims(P)
    with pytest.raises(H.HarmradError):
        g.adjoint_enable(True)
