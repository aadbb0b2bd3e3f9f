"""The cold-MHD back-up (Sec. 4.11) on the CUDA path, zone by zone through
the C ABI, against the oracle (tests/test_oracle_cold.py builds the zones:
flat space, no gas-radiation coupling, an explicit gas energy below the
kinetic energy of the motion, momentum-dominated radiation).

- harmrad_zone_implicit (no explicit entropy) and the no-allocation entry
  solve every zone with the cold-MHD equations: method HARMRAD_ZONE_COLD,
  u_g equal to the guess's, every primitive within 1e-10 of the oracle's
  (both Newton solves stop once e_T < 1e-12, Sec. 4.10, which leaves their
  roots up to about 1e-11 apart);
- harmrad_zone_implicit_full with the true state's entropy solves the zones
  with the entropy equation first (HARMRAD_ZONE_ENTROPY), without an explicit
  entropy (not finite) with the cold-MHD equations, and a zone whose
  radiation is not momentum-dominated takes the back-up (HARMRAD_ZONE_BACKUP),
  each as in the oracle; the entropy zones' u_g within 1e-10 of u_g plus the
  gas energy row |T^t_t + rho0 u^t| (the scale on which the entropy row,
  with its factor T and the energy norm of Sec. 4.8, fixes u_g of these cold
  zones), every other primitive within 1e-10 of the oracle's.

A grid step hands a cold-MHD zone's u_g to the neighbour average; no workload
here reaches that branch (it needs radiation with |F| > sqrt(10) E after the
explicit update), so it is not exercised on the GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_6127_gb300 import harmrad as H
from tests.test_oracle_cold import X, cold_cases

pytestmark = pytest.mark.gpu

RHO, UU, ER, UR1, UR3 = 0, 1, 8, 9, 11


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("B_amp", [0.0, 0.05])
def test_cold_zones_match_oracle(B_amp):
    cfg, cases = cold_cases(count=64, seed=3031, B_amp=B_amp)
    p = O.make_params(cfg)
    x = np.array([X] * len(cases))
    U = np.array([c[0] for c in cases])
    Ps = np.array([c[1] for c in cases])
    ref = [O.implicit_zone(p, X, U[k], Ps[k], 0.1) for k in range(len(cases))]
    assert all(r[1].cold == 1 for r in ref)
    Pg, eT, it, meth = H.zone_implicit(cfg, x, U, Ps, 0.1)
    assert np.all(meth == H.ZONE_COLD), np.bincount(meth)
    assert np.array_equal(Pg[:, UU], Ps[:, UU])
    err = max(_rel(Pg[k], ref[k][0]).max() for k in range(len(cases)))
    print("cold-MHD zones, B amplitude %.2f: worst relative error %.2e, e_T up to %.1e" % (B_amp, err, eT.max()))
    assert err < 1e-10 and eT.max() < 1e-12


def test_cold_zones_static_entry():
    import ctypes
    import torch

    cfg, cases = cold_cases(count=32, seed=3032)
    p = O.make_params(cfg)
    n = len(cases)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    U = np.array([c[0] for c in cases])
    Ps = np.array([c[1] for c in cases])
    xd, Ud, Pd, hd = dev([X] * n), dev(U), dev(Ps), dev(np.full(n, 0.1))
    Pout = torch.empty((n, 12), dtype=torch.float64, device="cuda")
    eT = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    me = torch.empty(n, dtype=torch.uint8, device="cuda")
    hp = H.make_params(cfg)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = H.load().harmrad_zone_implicit_static(ctypes.byref(hp), n, vp(xd), vp(Ud), vp(Pd), vp(hd), vp(Pout),
                                               vp(eT), vp(it), vp(me), stream)
    assert rc == 0
    meth, Pg = me.cpu().numpy(), Pout.cpu().numpy()
    assert np.all(meth == H.ZONE_COLD)
    err = max(_rel(Pg[k], O.implicit_zone(p, X, U[k], Ps[k], 0.1)[0]).max() for k in range(n))
    assert err < 1e-10, err


def test_backup_order_matches_oracle():
    cfg, cases = cold_cases(count=24, seed=3033)
    p = O.make_params(cfg)
    n_ad = 1.0 / (cfg["gam"] - 1.0)
    U, Ps, S, want = [], [], [], []
    for k, (u, ps, P) in enumerate(cases):
        kind = k % 3
        v = u.copy()
        if kind == 0:  # the true state's entropy: the entropy equation solves the zone
            s = v[RHO] * (n_ad * math.log((cfg["gam"] - 1.0) * P[UU]) - (n_ad + 1.0) * math.log(P[RHO]))
        elif kind == 1:  # no explicit entropy (not finite): the cold-MHD equations
            s = math.nan
        else:  # |F| = 2 E: not momentum-dominated, the back-up
            s = math.nan
            v[UR1:UR3 + 1] *= 2.0 * (-v[ER]) / np.linalg.norm(v[UR1:UR3 + 1])
        out, info = O.implicit_zone(p, X, v, ps, 0.1, Sstar=s)
        code = H.ZONE_ENTROPY if info.entropy else (H.ZONE_COLD if info.cold else info.method)
        U.append(v)
        Ps.append(ps)
        S.append(s)
        want.append((code, out))
    Pg, eT, it, meth = H.zone_implicit(cfg, np.array([X] * len(U)), np.array(U), np.array(Ps), 0.1,
                                       Sstar=np.array(S))
    codes = [w[0] for w in want]
    assert list(meth) == codes, (list(meth), codes)
    assert set(codes) == {H.ZONE_ENTROPY, H.ZONE_COLD, H.ZONE_BACKUP}
    for k, (code, out) in enumerate(want):
        if code != H.ZONE_BACKUP:
            r = _rel(Pg[k], out)
            if code == H.ZONE_ENTROPY:
                r[UU] = abs(Pg[k][UU] - out[UU]) / (out[UU] + abs(U[k][UU] / U[k][RHO]) * out[RHO])
            assert r.max() < 1e-10, (k, code, r.max())
