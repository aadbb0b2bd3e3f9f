"""Pins of the oracle's staggered magnetic field (Sec. 4: B on the cell faces,
EMFs on the edges; Sec. 4.2 steps viii-x: the 4-state upwind EMF after Del
Zanna et al. 2007).

- Constrained transport: each face changes by the curl of edge EMFs, so the
  face divergence sum_d (Bf_d(+) - Bf_d(-))/dx_d of every zone keeps its
  initial value to round-off, whatever the EMFs are; a sign or index slip in
  the face update breaks it.  Checked on a 3D periodic box with a random
  field from a vector potential and on the Kerr-Schild torus (outflow and
  polar boundaries).
- Consistency and order: a weak field from A_z = A0 sin(2 pi x) sin(2 pi y)
  carried by a uniform flow through a periodic box is the translated field
  (the field is too weak to act on the flow); the face field converges to it
  at second order, as the MC-limited interpolation of the scheme allows, and
  a wrong sign of a dissipation or EMF term spoils either the order or the
  stability.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import workloads as W


def face_div(Bf, dx):
    return ((Bf[0][:, :, 1:] - Bf[0][:, :, :-1]) / dx[0] + (Bf[1][:, 1:, :] - Bf[1][:, :-1, :]) / dx[1]
            + (Bf[2][1:] - Bf[2][:-1]) / dx[2])


def curl_faces(A, dx):
    """Face fields sqrt(-g) B = curl A of a periodic edge potential A[d]
    ([n3, n2, n1] each; A_1 on (i, j-1/2, k-1/2), A_2 on (i-1/2, j, k-1/2),
    A_3 on (i-1/2, j-1/2, k)), with the periodic image face appended."""
    up = lambda a, ax: np.roll(a, -1, axis=ax)
    B1 = (up(A[2], 1) - A[2]) / dx[1] - (up(A[1], 0) - A[1]) / dx[2]
    B2 = (up(A[0], 0) - A[0]) / dx[2] - (up(A[2], 2) - A[2]) / dx[0]
    B3 = (up(A[1], 2) - A[1]) / dx[0] - (up(A[0], 1) - A[0]) / dx[1]
    pad = lambda b, ax: np.concatenate([b, b.take([0], axis=ax)], axis=ax)
    return [pad(B1, 2), pad(B2, 1), pad(B3, 0)]


@pytest.mark.parametrize("recon,flux", [(W.PPM, W.LAXF), (W.MC, W.HLL)])
def test_face_divergence_box(recon, flux):
    cfg, P = W.minkowski_box((12, 10, 8), seed=3, recon=recon, flux=flux)
    cfg["emf"] = 1
    o = O.Oracle(cfg)
    o.set_prims(P)
    g = W.rng(5)
    A = [0.05 * g.standard_normal((8, 10, 12)) for _ in range(3)]
    o.set_face_fields(curl_faces(A, cfg["dx"]))
    b0 = o.get_face_fields()
    scale = max(np.abs(b).max() for b in b0) / min(cfg["dx"])
    d0 = face_div(b0, cfg["dx"])
    for _ in range(4):
        o.step(0.0)
    b = o.get_face_fields()
    change = max(np.abs(b[i] - b0[i]).max() for i in range(3))
    drift = np.abs(face_div(b, cfg["dx"]) - d0).max()
    print("box: field change %.2e, divergence drift %.2e of scale %.2e" % (change, drift, scale))
    assert change > 1e-2
    assert drift < 1e-14 * scale


def test_face_divergence_torus():
    cfg, P, Bf = W.torus((16, 8, 4), faces=True)
    cfg["emf"] = 1
    o = O.Oracle(cfg)
    o.set_prims(P)
    o.set_face_fields(Bf)
    np.testing.assert_allclose(o.get_prims()[5:8], P[5:8], rtol=1e-12, atol=1e-15 * np.abs(P[5:8]).max())
    b0 = o.get_face_fields()
    scale = max(np.abs(b).max() for b in b0) / min(cfg["dx"])
    d0 = face_div(b0, cfg["dx"])
    assert np.abs(d0).max() < 1e-15 * scale
    for _ in range(3):
        o.step(0.0)
    b = o.get_face_fields()
    drift = np.abs(face_div(b, cfg["dx"]) - d0).max()
    print("torus: divergence drift %.2e of scale %.2e" % (drift, scale))
    assert drift < 1e-14 * scale
    # the polar faces carry no flux
    assert np.all(b[1][:, 0, :] == 0.0) and np.all(b[1][:, -1, :] == 0.0)


def advect(n, T, A0=1e-4, v=(0.2, 0.1)):
    """Relative L1 error of the x-face field after time T against the
    translated initial field."""
    cfg = W.base_params()
    cfg.update(n=[n, n, 1], dx=[1.0 / n, 1.0 / n, 1.0], recon=W.MC, flux=W.HLL, emf=1, a_rad=1e-6,
               floor_rho0=1e-12, floor_u0=1e-14)
    gam = 1.0 / math.sqrt(1.0 - v[0] ** 2 - v[1] ** 2)
    P = np.zeros((12, 1, n, n))
    P[0] = 1.0
    P[1] = 1.0
    P[2] = gam * v[0]
    P[3] = gam * v[1]
    P[8] = 1e-8
    xe = np.arange(n) / n

    def faces(t):
        X, Y = np.meshgrid(xe - v[0] * t, xe - v[1] * t)  # edges (i-1/2, j-1/2) at [j, i]
        A3 = A0 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
        return curl_faces([np.zeros((1, n, n)), np.zeros((1, n, n)), A3[None]], cfg["dx"])

    o = O.Oracle(cfg)
    o.set_prims(P)
    o.set_face_fields(faces(0.0))
    t = 0.0
    while t < T - 1e-12:
        dt = min(o.cfl_dt(), T - t)
        o.step(dt)
        t += dt
    b, ex = o.get_face_fields()[0], faces(T)[0]
    return np.abs(b - ex).mean() / np.abs(ex).mean()


def test_field_advection_second_order():
    e1, e2 = advect(16, 1.25), advect(32, 1.25)
    order = math.log2(e1 / e2)
    print("advected field: L1 errors %.3e (16^2), %.3e (32^2), order %.2f" % (e1, e2, order))
    assert order > 1.7 and e2 < 0.05
