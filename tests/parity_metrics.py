"""Per-zone error measures used by the GPU parity tests.

rho0 is compared relative to its own value.  u_g and Ebar are compared
relative to their own value plus 1e-2 of the zone's energy-row scale
|T^t_t + rho0 u^t| (the quantity the implicit solve's e_T < 1e-12 test
normalises by), so that an error below 1e-10 means
|du| <= 1e-10 u + 1e-12 |T^t_t + rho0 u^t|: agreement to the Newton tolerance
of Sec. 4.10.  Signed components are compared against the physical scale of
their group, because a component that is zero by symmetry carries only
round-off:
  - gas velocity u~^i: |du~^i| sqrt(g_ii) / (|u~| + c_s), c_s the local sound
    speed, |u~| = sqrt(g_ij u~^i u~^j);
  - radiation-frame velocity: |du~^i_rad| sqrt(g_ii) / (|u~_rad| + 1/sqrt(3));
  - field B^i: |dB^i| sqrt(g_ii) / (|B| + sqrt(2 p_g)), |B| = sqrt(g_ij B^i B^j).
Fluxes are compared per component against |F| + 1e-3 S, S the largest flux
of the component's group (mass; gas energy-momentum; induction; radiation)
over all directions: an error below 1e-10 means |dF| <= 1e-10 |F| + 1e-13 S.
"""
import numpy as np

from oracle import oracle as O

GROUPS = [(0,), (1, 2, 3, 4), (5, 6, 7), (8, 9, 10, 11)]


def _metric_diag(cfg, shape):
    """sqrt(g_ii) (i = 1..3) at the zone centres, from the oracle's metric."""
    n3, n2, n1 = shape
    out = np.ones((3,) + shape)
    p = O.make_params(cfg)
    x1 = [cfg["x0"][0] + (i + 0.5) * cfg["dx"][0] for i in range(n1)]
    x2 = [cfg["x0"][1] + (j + 0.5) * cfg["dx"][1] for j in range(n2)]
    G = np.zeros((n2, n1, 4, 4))
    for j in range(n2):
        for i in range(n1):
            G[j, i] = O.metric(p, [0.0, x1[i], x2[j], 0.0])[0]
    for d in range(3):
        out[d] = np.sqrt(G[:, :, d + 1, d + 1])[None, :, :]
    return out, G


def _vec_mag(G, v):
    # sqrt(g_ij v^i v^j) with G[j, i, 4, 4] broadcast over k
    s = np.zeros(v.shape[1:])
    for a in range(3):
        for b in range(3):
            s += G[None, :, :, a + 1, b + 1] * v[a] * v[b]
    return np.sqrt(np.maximum(s, 0.0))


def zone_errors(cfg, A, R):
    """Per-zone, per-primitive errors of A against the reference R ([12,n3,n2,n1])."""
    shape = R.shape[1:]
    if cfg["metric"] == 0:
        sg = np.ones((3,) + shape)
        G = np.zeros((shape[1], shape[2], 4, 4))
        for d in range(4):
            G[:, :, d, d] = 1.0 if d else -1.0
    else:
        sg, G = _metric_diag(cfg, shape)
    E = np.zeros_like(R)
    escale = energy_scale(cfg, R)
    E[0] = np.abs(A[0] - R[0]) / np.abs(R[0])
    for q in (1, 8):
        E[q] = np.abs(A[q] - R[q]) / (np.abs(R[q]) + 1e-2 * escale)
    gam = cfg["gam"]
    pg = (gam - 1.0) * R[1]
    cs = np.sqrt(gam * pg / (R[0] + R[1] + pg))
    ug = _vec_mag(G, R[2:5]) + cs
    ur = _vec_mag(G, R[9:12]) + 1.0 / np.sqrt(3.0)
    bs = _vec_mag(G, R[5:8]) + np.sqrt(2.0 * pg)
    for i in range(3):
        E[2 + i] = np.abs(A[2 + i] - R[2 + i]) * sg[i] / ug
        E[5 + i] = np.abs(A[5 + i] - R[5 + i]) * sg[i] / bs
        E[9 + i] = np.abs(A[9 + i] - R[9 + i]) * sg[i] / ur
    return E


def plain_relative(A, R):
    """Plain relative errors |A - R| / |R| of u_g and Ebar per zone (the
    unconditioned companions of the per-zone measure above), as (max, p99)
    of each."""
    out = {}
    for q, name in ((1, "u_g"), (8, "Ebar")):
        e = (np.abs(A[q] - R[q]) / np.abs(R[q])).ravel()
        out[name] = (float(e.max()), float(np.quantile(e, 0.99)))
    return out


def energy_scale(cfg, R):
    """|T^t_t + rho0 u^t| per zone from the oracle's conserved variables."""
    p = O.make_params(cfg)
    n3, n2, n1 = R.shape[1:]
    out = np.empty((n3, n2, n1))
    for k in range(n3):
        for j in range(n2):
            for i in range(n1):
                x = [0.0, cfg["x0"][0] + (i + 0.5) * cfg["dx"][0],
                     cfg["x0"][1] + (j + 0.5) * cfg["dx"][1], cfg["x0"][2] + (k + 0.5) * cfg["dx"][2]]
                gd = O.metric(p, x)[2]
                U, _ = O.prim_to_cons(p, x, R[:, k, j, i])
                out[k, j, i] = abs(U[1]) / gd
    return out


def group_scales(Fo_all):
    """Largest flux of each group over all directions (list of [12,...] arrays)."""
    return [max(max(np.abs(F[list(grp)]).max() for F in Fo_all), 1e-300) for grp in GROUPS]


def flux_errors(Fg, Fo, scales=None):
    if scales is None:
        scales = group_scales([Fo])
    E = np.zeros_like(Fo)
    for grp, sc in zip(GROUPS, scales):
        for q in grp:
            E[q] = np.abs(Fg[q] - Fo[q]) / (np.abs(Fo[q]) + 1e-3 * sc)
    return E


def point_errors(metric_cfg, x, A, R, gam, rad_conserved=False):
    """Errors of point states A vs R ([12] each) at internal position x.

    rad_conserved: measure the radiation (entries 8..11) in conserved form,
    |dR^t_nu| (orthonormal ZAMO size for the spatial components) against
    |R^t_t| + |T^t_t + rho0 u^t|.  The PMHD solve recovers the radiation from
    total energy-momentum conservation, so its absolute precision is set by the
    total energy scale, and a sub-dominant radiation field carries that error
    relative to its own, smaller, primitives."""
    p = O.make_params(metric_cfg)
    gcov = O.metric(p, x)[0]
    sg = np.sqrt(np.diag(gcov)[1:])
    Gs = gcov[1:, 1:]
    mag = lambda v: np.sqrt(max(v @ Gs @ v, 0.0))
    e = np.zeros(12)
    gd = O.metric(p, x)[2]
    U, _ = O.prim_to_cons(p, x, R)
    escale = abs(U[1]) / gd
    e[0] = abs(A[0] - R[0]) / abs(R[0])
    for q in (1, 8):
        e[q] = abs(A[q] - R[q]) / (abs(R[q]) + 1e-2 * escale)
    pg = (gam - 1.0) * R[1]
    cs = np.sqrt(gam * pg / (R[0] + R[1] + pg))
    ug = mag(R[2:5]) + cs
    ur = mag(R[9:12]) + 1.0 / np.sqrt(3.0)
    bs = mag(R[5:8]) + np.sqrt(2.0 * pg)
    for i in range(3):
        e[2 + i] = abs(A[2 + i] - R[2 + i]) * sg[i] / ug
        e[5 + i] = abs(A[5 + i] - R[5 + i]) * sg[i] / bs
        e[9 + i] = abs(A[9 + i] - R[9 + i]) * sg[i] / ur
    if rad_conserved:
        gcon = O.metric(p, x)[1]
        UA, _ = O.prim_to_cons(p, x, A)
        scale = abs(U[8]) + abs(U[1])
        e[8] = abs(UA[8] - U[8]) / scale
        for i in range(3):
            zi = np.sqrt(gcon[i + 1, i + 1] - gcon[0, i + 1] ** 2 / gcon[0, 0])
            e[9 + i] = abs(UA[9 + i] - U[9 + i]) * zi / scale
    return e
