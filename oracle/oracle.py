"""ctypes wrapper of the HARMRAD FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The oracle is a plain restatement of
the time step of McKinney et al. (2014), Sec. 4, written independently of the
CUDA library; see ``oracle.h`` for the conventions.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["oracle_phys.cpp", "oracle_implicit.cpp", "oracle_grid.cpp"]
_HDR = ["oracle.h", "oracle_internal.h"]
_LIB = os.path.join(_HERE, "liboracle.so")

NP = 12
RHO, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3 = range(12)
OK_PMHD, OK_URAD, BACKUP = 0, 1, 2


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("x0", ctypes.c_double * 3),
        ("dx", ctypes.c_double * 3),
        ("metric", ctypes.c_int),
        ("a_spin", ctypes.c_double),
        ("R0", ctypes.c_double),
        ("hslope", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("gam", ctypes.c_double),
        ("a_rad", ctypes.c_double),
        ("courant", ctypes.c_double),
        ("opacity", ctypes.c_int),
        ("kappa_abs0", ctypes.c_double),
        ("kappa_es0", ctypes.c_double),
        ("kappa_scale", ctypes.c_double),
        ("T_kappa_min", ctypes.c_double),
        ("recon", ctypes.c_int),
        ("flux", ctypes.c_int),
        ("gamma_rad_max", ctypes.c_double),
        ("gamma_gas_max", ctypes.c_double),
        ("floor_rho0", ctypes.c_double),
        ("floor_rho_pow", ctypes.c_double),
        ("floor_u0", ctypes.c_double),
        ("floor_u_pow", ctypes.c_double),
        ("bsq_rho_max", ctypes.c_double),
        ("bsq_u_max", ctypes.c_double),
        ("u_rho_max", ctypes.c_double),
        ("newton_max", ctypes.c_int),
        ("newton_tol", ctypes.c_double),
        ("integrator", ctypes.c_int),
        ("implicit_eq", ctypes.c_int),
        ("emf", ctypes.c_int),
    ]


class OrcInfo(ctypes.Structure):
    _fields_ = [
        ("e_T", ctypes.c_double),
        ("iters_pmhd", ctypes.c_int),
        ("iters_urad", ctypes.c_int),
        ("method", ctypes.c_int),
        ("neg_erad", ctypes.c_int),
        ("entropy", ctypes.c_int),
        ("cold", ctypes.c_int),
    ]


def build(force=False):
    """Compile the oracle with g++ (plain -O2, no FMA contraction; OpenMP
    for the zone and face loops, ORACLE_THREADS threads, default 1)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDR]
    if not force and os.path.exists(_LIB):
        t = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= t for s in deps):
            return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OrcParams)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [pp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_prims.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_prims.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_opacity_field.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_prims_with_ghosts.argtypes = [ctypes.c_void_p, dp, ctypes.c_int]
        L.orc_set_prims_with_ghosts.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_face_fields.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_face_fields.argtypes = [ctypes.c_void_p, dp]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [ctypes.c_void_p]
        L.orc_step.restype = ctypes.c_double
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_get_status.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ubyte)]
        L.orc_get_iters.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
        L.orc_get_counts.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_compute_fluxes.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.orc_metric.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_connection.argtypes = [pp, dp, dp]
        L.orc_prim_to_cons.argtypes = [pp, dp, dp, dp, dp]
        L.orc_flux.argtypes = [pp, dp, ctypes.c_int, dp, dp, dp]
        L.orc_stress.argtypes = [pp, dp, dp, dp, dp]
        L.orc_four_force.argtypes = [pp, dp, dp, dp]
        L.orc_rad_invert.restype = ctypes.c_int
        L.orc_rad_invert.argtypes = [pp, dp, dp, ctypes.c_int, dp]
        L.orc_gas_invert.restype = ctypes.c_int
        L.orc_gas_invert.argtypes = [pp, dp, dp, dp, ctypes.c_double, dp]
        L.orc_implicit_zone.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, dp, ctypes.POINTER(OrcInfo)]
        L.orc_radiation_subdominant.argtypes = [pp, dp, dp, dp]
        L.orc_cold_allowed.argtypes = [pp, dp, dp, dp]
        L.orc_cold_allowed.restype = ctypes.c_int
        L.orc_method_zone.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp, dp,
                                      ctypes.POINTER(ctypes.c_int)]
        L.orc_radiation_subdominant.restype = ctypes.c_int
        L.orc_pmhd_residual.argtypes = [pp, dp, dp, ctypes.c_double, dp, dp, dp, dp]
        L.orc_face_flux_stencil.argtypes = [pp, ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_apply_floors.argtypes = [pp, dp, dp]
        L.orc_ppm_cell.argtypes = [dp, ctypes.c_double, dp, dp]
        L.orc_mc_slope.restype = ctypes.c_double
        L.orc_mc_slope.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_levermore_xi.restype = ctypes.c_double
        L.orc_levermore_xi.argtypes = [ctypes.c_double]
    return _lib


def make_params(cfg):
    """Fill an OrcParams from a plain dict of configuration values."""
    p = OrcParams()
    for name, ctype in OrcParams._fields_:
        if name not in cfg:
            raise KeyError("missing parameter %s" % name)
        v = cfg[name]
        if hasattr(ctype, "_length_"):
            arr = getattr(p, name)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, name, v)
    return p


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


class Oracle:
    """Grid-level oracle: owns one grid, steps it on the host."""

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self.p = make_params(cfg)
        self.n = tuple(cfg["n"])
        self._h = lib().orc_create(ctypes.byref(self.p))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (NP, self.n[2], self.n[1], self.n[0])

    def set_prims(self, P):
        P = _vec(P).reshape(self.shape)
        lib().orc_set_prims(self._h, _dp(P))

    def set_opacity_field(self, K):
        """Absorption field of opacity mode 2 ([n3,n2,n1]; per length kappa_scale K)."""
        K = _vec(K).reshape(self.shape[1:])
        lib().orc_set_opacity_field(self._h, _dp(K))

    def get_prims(self):
        P = np.empty(self.shape)
        lib().orc_get_prims(self._h, _dp(P))
        return P

    def cfl_dt(self):
        return lib().orc_cfl_dt(self._h)

    def step(self, dt=0.0):
        return lib().orc_step(self._h, float(dt))

    def status(self):
        st = np.empty(self.shape[1:], dtype=np.uint8)
        lib().orc_get_status(self._h, st.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return st

    def iters(self):
        it = np.empty(self.shape[1:], dtype=np.int32)
        lib().orc_get_iters(self._h, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return it

    def counts(self):
        c = np.zeros(7, dtype=np.int64)
        lib().orc_get_counts(self._h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        return {"pmhd": int(c[0]), "urad": int(c[1]), "backup": int(c[2]),
                "iters": int(c[3]), "solves": int(c[4]), "entropy": int(c[5]), "cold": int(c[6])}

    def fluxes(self, d):
        m = list(self.n)
        m[d - 1] += 1
        F = np.empty((NP, m[2], m[1], m[0]))
        lib().orc_compute_fluxes(self._h, d, _dp(F))
        return F

    def face_shapes(self):
        """Shapes [n3', n2', n1'] of the three face-field arrays (staggered field)."""
        out = []
        for d in range(3):
            m = list(self.n)
            if m[d] > 1:
                m[d] += 1
            out.append((m[2], m[1], m[0]))
        return out

    def set_face_fields(self, Bf):
        """sqrt(-g) B^d on the d-faces (three arrays of face_shapes())."""
        flat = np.concatenate([np.ascontiguousarray(b, dtype=np.float64).ravel() for b in Bf])
        lib().orc_set_face_fields(self._h, _dp(flat))

    def get_face_fields(self):
        shapes = self.face_shapes()
        flat = np.empty(sum(int(np.prod(s)) for s in shapes))
        lib().orc_get_face_fields(self._h, _dp(flat))
        out, off = [], 0
        for s in shapes:
            m = int(np.prod(s))
            out.append(flat[off:off + m].reshape(s))
            off += m
        return out

    def set_prims_with_ghosts(self, P):
        """Every cell, ghosts included ([12, N3, N2, N1]); fixed faces keep their ghosts."""
        ng = [4 if x > 1 else 0 for x in self.n]
        N = [self.n[i] + 2 * ng[i] for i in range(3)]
        P = _vec(P).reshape((NP, N[2], N[1], N[0]))
        lib().orc_set_prims_with_ghosts(self._h, _dp(P))

    def prims_with_ghosts(self, fill=True):
        ng = [4 if x > 1 else 0 for x in self.n]
        N = [self.n[i] + 2 * ng[i] for i in range(3)]
        P = np.empty((NP, N[2], N[1], N[0]))
        lib().orc_get_prims_with_ghosts(self._h, _dp(P), 1 if fill else 0)
        return P


# ---- point-wise physics ----------------------------------------------------

def metric(p, x):
    x = _vec(x)
    gcov = np.empty(16)
    gcon = np.empty(16)
    gdet = ctypes.c_double()
    alpha = ctypes.c_double()
    lib().orc_metric(ctypes.byref(p), _dp(x), _dp(gcov), _dp(gcon), ctypes.byref(gdet),
                     ctypes.byref(alpha))
    return gcov.reshape(4, 4), gcon.reshape(4, 4), gdet.value, alpha.value


def connection(p, x):
    x = _vec(x)
    g = np.empty(64)
    lib().orc_connection(ctypes.byref(p), _dp(x), _dp(g))
    return g.reshape(4, 4, 4)


def prim_to_cons(p, x, P):
    x, P = _vec(x), _vec(P)
    U = np.empty(NP)
    SM = np.empty(NP)
    lib().orc_prim_to_cons(ctypes.byref(p), _dp(x), _dp(P), _dp(U), _dp(SM))
    return U, SM


def flux(p, x, d, P):
    x, P = _vec(x), _vec(P)
    F = np.empty(NP)
    sp = np.empty(4)
    lib().orc_flux(ctypes.byref(p), _dp(x), int(d), _dp(P), _dp(F), _dp(sp))
    return F, sp


def stress(p, x, P):
    x, P = _vec(x), _vec(P)
    T = np.empty(16)
    R = np.empty(16)
    lib().orc_stress(ctypes.byref(p), _dp(x), _dp(P), _dp(T), _dp(R))
    return T.reshape(4, 4), R.reshape(4, 4)


def four_force(p, x, P):
    x, P = _vec(x), _vec(P)
    G = np.empty(4)
    lib().orc_four_force(ctypes.byref(p), _dp(x), _dp(P), _dp(G))
    return G


def rad_invert(p, x, Rt, limiter=2):
    x, Rt = _vec(x), _vec(Rt)
    out = np.empty(4)
    neg = lib().orc_rad_invert(ctypes.byref(p), _dp(x), _dp(Rt), int(limiter), _dp(out))
    return out, neg


def gas_invert(p, x, U, Pg, tol=1e-14):
    x, U, Pg = _vec(x), _vec(U), _vec(Pg)
    out = np.empty(NP)
    rc = lib().orc_gas_invert(ctypes.byref(p), _dp(x), _dp(U), _dp(Pg), float(tol), _dp(out))
    return out, rc


def implicit_zone(p, x, Ustar, Ps, h, Sstar=None):
    """Implicit solve of one zone; Sstar = sqrt(-g) S u^t of the explicit
    update enables the entropy back-up (None: energy methods, then the
    cold-MHD equations)."""
    x, Ustar, Ps = _vec(x), _vec(Ustar), _vec(Ps)
    out = np.empty(NP)
    info = OrcInfo()
    sp = None
    if Sstar is not None:
        sv = ctypes.c_double(float(Sstar))
        sp = ctypes.pointer(sv)
    lib().orc_implicit_zone(ctypes.byref(p), _dp(x), _dp(Ustar), sp, _dp(Ps), float(h), _dp(out),
                            ctypes.byref(info))
    return out, info


def method_zone(p, x, Ustar, Ps, h, method, Sstar=None):
    """One Newton method alone (0 PMHD, 1 URAD, 2 PRAD, 3 staged PMHD with
    u_g from the explicit entropy Sstar if given, 4 staged URAD, 5 staged
    PRAD, 6/7/8 the entropy-based PMHD/URAD/PRAD with the explicit entropy
    Sstar): (P, e_T, steps)."""
    x, Us, Pz = _vec(x), _vec(Ustar), _vec(Ps)
    out = np.empty(NP)
    eT = ctypes.c_double()
    it = ctypes.c_int()
    sp = None
    if Sstar is not None:
        sv = ctypes.c_double(float(Sstar))
        sp = ctypes.pointer(sv)
    lib().orc_method_zone(ctypes.byref(p), _dp(x), _dp(Us), sp, _dp(Pz), float(h), int(method), _dp(out),
                          ctypes.byref(eT), ctypes.byref(it))
    return out, eT.value, it.value


def radiation_subdominant(p, x, Ustar, Ps):
    """Sec. 4.10 sub-dominance test of one zone."""
    x, Us, Pz = _vec(x), _vec(Ustar), _vec(Ps)
    return bool(lib().orc_radiation_subdominant(ctypes.byref(p), _dp(x), _dp(Us), _dp(Pz)))


def cold_allowed(p, x, Ustar, Ps):
    """Sec. 4.11 test of one zone for the cold-MHD back-up."""
    x, Us, Pz = _vec(x), _vec(Ustar), _vec(Ps)
    return bool(lib().orc_cold_allowed(ctypes.byref(p), _dp(x), _dp(Us), _dp(Pz)))


def pmhd_residual(p, x, Ustar, h, xg):
    x, Ustar, xg = _vec(x), _vec(Ustar), _vec(xg)
    E = np.empty(4)
    eT = ctypes.c_double()
    eI = ctypes.c_double()
    lib().orc_pmhd_residual(ctypes.byref(p), _dp(x), _dp(Ustar), float(h), _dp(xg), _dp(E),
                            ctypes.byref(eT), ctypes.byref(eI))
    return E, eT.value, eI.value


def face_flux_stencil(p, d, S, xc, xf):
    """Flux of one face of direction d from its 8-cell stencil S[8][12]."""
    S, xc, xf = _vec(S), _vec(xc), _vec(xf)
    F = np.empty(NP)
    sp = ctypes.c_double()
    lib().orc_face_flux_stencil(ctypes.byref(p), int(d), _dp(S), _dp(xc), _dp(xf), _dp(F), ctypes.byref(sp))
    return F, sp.value


def apply_floors(p, x, P):
    """The grid step's floors applied to one zone's primitives (copy returned)."""
    Q = _vec(P).copy()
    lib().orc_apply_floors(ctypes.byref(p), _dp(_vec(x)), _dp(Q))
    return Q


def ppm_cell(s5, chi=0.0):
    """PPM edge values (aL, aR) of the centre cell of a 5-cell stencil."""
    s = _vec(s5)
    aL, aR = ctypes.c_double(), ctypes.c_double()
    lib().orc_ppm_cell(_dp(s), float(chi), ctypes.byref(aL), ctypes.byref(aR))
    return aL.value, aR.value


def mc_slope(qm, q0, qp):
    return lib().orc_mc_slope(float(qm), float(q0), float(qp))


def levermore_xi(f):
    return lib().orc_levermore_xi(float(f))
