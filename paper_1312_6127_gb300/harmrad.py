"""Python binding of the harmrad C ABI (include/harmrad.h).

Argument marshalling only: every step of the time step runs in the CUDA
kernels of ``libharmrad.so``.  PyTorch provides device memory and the CUDA
stream.  Importing works without a GPU; creating a grid or calling a kernel
requires the built library and a CUDA device, and raises otherwise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libharmrad.so")
NPRIM = 12

OK, W_BACKUP_USED = 0, 1
ZONE_PMHD, ZONE_URAD, ZONE_BACKUP, ZONE_ENTROPY, ZONE_COLD = 0, 1, 2, 3, 4
PREC_FP64, PREC_SPLIT = 0, 1
OPAC_CONST, OPAC_KRAMERS, OPAC_FIELD = 0, 1, 2
INT_RK3, INT_IMEX2, INT_IMEX2B, INT_IMEX3 = 0, 1, 2, 3
EQ_ENERGY, EQ_ENTROPY = 0, 1
EMF_FLUXCT, EMF_UCT = 0, 1

EXPORTS = [
    "harmrad_init", "harmrad_init_batch", "harmrad_destroy", "harmrad_set_opacity_field", "harmrad_set_prims",
    "harmrad_set_prims_ghosts", "harmrad_get_prims", "harmrad_set_face_fields", "harmrad_get_face_fields",
    "harmrad_cfl_dt", "harmrad_step", "harmrad_step_host", "harmrad_get_stats",
    "harmrad_get_status", "harmrad_get_iters", "harmrad_compute_fluxes",
    "harmrad_zone_physics", "harmrad_zone_implicit", "harmrad_zone_implicit_full", "harmrad_zone_method",
    "harmrad_zone_implicit_static",
    "harmrad_profile_step", "harmrad_autotune", "harmrad_get_tuning", "harmrad_set_tuning",
    "harmrad_adjoint_enable", "harmrad_step_adjoint", "harmrad_adjoint_set_input",
    "harmrad_branch_signature", "harmrad_get_branch_signature",
    "harmrad_fp64_fma_rate",
    "harmrad_strerror",
]
KERNEL_CLASSES = ["bc", "prep", "flatten", "face", "ct", "update", "retry", "backup", "cfl", "other",
                  "edge"]


class Params(ctypes.Structure):
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
        ("precision", ctypes.c_int),
        ("integrator", ctypes.c_int),
        ("implicit_eq", ctypes.c_int),
        ("emf", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double),
        ("zone_stages", ctypes.c_longlong),
        ("pmhd_ok", ctypes.c_longlong),
        ("urad_ok", ctypes.c_longlong),
        ("backup", ctypes.c_longlong),
        ("newton_iters", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_int),
        ("graph", ctypes.c_int),
        ("entropy_ok", ctypes.c_longlong),
        ("cold_ok", ctypes.c_longlong),
    ]


class KernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 11), ("launches", ctypes.c_int * 11),
                ("total_launches", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("face_block", ctypes.c_int), ("face_blocks_per_sm", ctypes.c_int),
        ("update_block", ctypes.c_int), ("update_blocks_per_sm", ctypes.c_int),
        ("edge_block", ctypes.c_int), ("edge_blocks_per_sm", ctypes.c_int),
        ("newton_split", ctypes.c_int),
        ("face_ms", ctypes.c_double), ("update_ms", ctypes.c_double), ("edge_ms", ctypes.c_double),
    ]


class HarmradError(RuntimeError):
    pass


_lib = None


def load(path=LIB_PATH):
    """Load libharmrad.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HarmradError("libharmrad.so not found at %s: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    pp = ctypes.POINTER(Params)
    L.harmrad_init.argtypes = [pp, vp, ctypes.POINTER(vp)]
    L.harmrad_init_batch.argtypes = [pp, ip, vp, ctypes.POINTER(vp)]
    L.harmrad_set_opacity_field.argtypes = [vp, vp, ip]
    L.harmrad_destroy.argtypes = [vp]
    L.harmrad_destroy.restype = None
    L.harmrad_set_prims.argtypes = [vp, vp, ip]
    L.harmrad_set_prims_ghosts.argtypes = [vp, vp, ip]
    L.harmrad_get_prims.argtypes = [vp, vp, ip]
    L.harmrad_set_face_fields.argtypes = [vp, vp, ip]
    L.harmrad_get_face_fields.argtypes = [vp, vp, ip]
    L.harmrad_cfl_dt.argtypes = [vp, dp]
    L.harmrad_step.argtypes = [vp, ctypes.c_double]
    L.harmrad_step_host.argtypes = [vp, vp, vp, ctypes.c_double]
    L.harmrad_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.harmrad_get_status.argtypes = [vp, vp, ip]
    L.harmrad_get_iters.argtypes = [vp, vp, ip]
    L.harmrad_compute_fluxes.argtypes = [vp, ip, vp]
    L.harmrad_zone_physics.argtypes = [pp, ip, vp, vp, vp, vp, vp, vp, vp]
    L.harmrad_zone_implicit.argtypes = [pp, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.harmrad_zone_implicit_full.argtypes = [pp, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.harmrad_zone_method.argtypes = [pp, ip, vp, vp, vp, vp, vp, ip, vp, vp, vp, vp]
    L.harmrad_zone_implicit_static.argtypes = [pp, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.harmrad_profile_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(KernelTimes)]
    L.harmrad_adjoint_enable.argtypes = [vp, ip]
    L.harmrad_step_adjoint.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ip]
    L.harmrad_autotune.argtypes = [vp, ip, ctypes.POINTER(Tuning)]
    L.harmrad_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.harmrad_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.harmrad_adjoint_set_input.argtypes = [vp, vp, ctypes.c_double, ip]
    L.harmrad_branch_signature.argtypes = [vp, ip]
    L.harmrad_get_branch_signature.argtypes = [vp, vp, ip]
    L.harmrad_fp64_fma_rate.argtypes = [ip, dp, vp]
    L.harmrad_strerror.restype = ctypes.c_char_p
    L.harmrad_strerror.argtypes = [ip]
    _lib = L
    return L


def _check(rc, what):
    if rc < 0:
        raise HarmradError("%s failed: %s (%d)" % (what, load().harmrad_strerror(rc).decode(), rc))
    return rc


def make_params(cfg, precision=None):
    p = Params()
    for name, ctype in Params._fields_:
        if name == "precision":
            v = cfg.get("precision", PREC_FP64) if precision is None else precision
        elif name == "integrator":
            v = cfg.get("integrator", INT_RK3)
        else:
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


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Grid:
    """One grid on the current CUDA device, stepped by the library."""

    def __init__(self, cfg, precision=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise HarmradError("a CUDA device is required")
        L = load()
        self.cfg = dict(cfg)
        self.params = make_params(cfg, precision)
        self.n = tuple(cfg["n"])
        self.shape = (NPRIM, self.n[2], self.n[1], self.n[0])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(L.harmrad_init(ctypes.byref(self.params), _stream_ptr(self.stream), ctypes.byref(h)),
               "harmrad_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().harmrad_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_prims(self, P):
        """P: numpy float64 array (host) or torch CUDA float64 tensor, [12,n3,n2,n1]."""
        import torch
        if isinstance(P, torch.Tensor):
            assert P.is_cuda and P.dtype == torch.float64 and tuple(P.shape) == self.shape
            P = P.contiguous()
            _check(load().harmrad_set_prims(self._h, ctypes.c_void_p(P.data_ptr()), 1), "set_prims")
        else:
            P = np.ascontiguousarray(P, dtype=np.float64).reshape(self.shape)
            _check(load().harmrad_set_prims(self._h, P.ctypes.data_as(ctypes.c_void_p), 0), "set_prims")

    def set_prims_ghosts(self, P):
        """Every cell, ghosts included ([12, N3, N2, N1], numpy); the ghosts of
        HARMRAD_BC_FIXED faces keep these values."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        _check(load().harmrad_set_prims_ghosts(self._h, P.ctypes.data_as(ctypes.c_void_p), 0),
               "set_prims_ghosts")

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
        """sqrt(-g) B^d on the d-faces: three arrays of face_shapes()."""
        flat = np.concatenate([np.ascontiguousarray(b, dtype=np.float64).ravel() for b in Bf])
        _check(load().harmrad_set_face_fields(self._h, flat.ctypes.data_as(ctypes.c_void_p), 0), "set_face_fields")

    def get_face_fields(self):
        shapes = self.face_shapes()
        flat = np.empty(sum(int(np.prod(s)) for s in shapes))
        _check(load().harmrad_get_face_fields(self._h, flat.ctypes.data_as(ctypes.c_void_p), 0), "get_face_fields")
        out, off = [], 0
        for s in shapes:
            m = int(np.prod(s))
            out.append(flat[off:off + m].reshape(s))
            off += m
        return out

    def set_opacity_field(self, K):
        """Per-zone absorption field K ([n3,n2,n1]; kappa_abs = kappa_scale K)."""
        K = np.ascontiguousarray(K, dtype=np.float64).reshape(self.shape[1:])
        _check(load().harmrad_set_opacity_field(self._h, K.ctypes.data_as(ctypes.c_void_p), 0),
               "set_opacity_field")

    def get_prims(self, device=False):
        import torch
        if device:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
            _check(load().harmrad_get_prims(self._h, ctypes.c_void_p(out.data_ptr()), 1), "get_prims")
            return out
        out = np.empty(self.shape)
        _check(load().harmrad_get_prims(self._h, out.ctypes.data_as(ctypes.c_void_p), 0), "get_prims")
        return out

    def cfl_dt(self):
        dt = ctypes.c_double()
        _check(load().harmrad_cfl_dt(self._h, ctypes.byref(dt)), "cfl_dt")
        return dt.value

    def step(self, dt=0.0):
        _check(load().harmrad_step(self._h, float(dt)), "step")

    def step_host(self, P_in, P_out, dt=0.0):
        """Host-in, host-out step through the C ABI (both numpy float64)."""
        _check(load().harmrad_step_host(self._h, P_in.ctypes.data_as(ctypes.c_void_p),
                                        P_out.ctypes.data_as(ctypes.c_void_p), float(dt)), "step_host")

    def profile_step(self, dt=0.0):
        """One eager step with an event after every kernel: per-class device ms."""
        kt = KernelTimes()
        _check(load().harmrad_profile_step(self._h, float(dt), ctypes.byref(kt)), "profile_step")
        return {name: (kt.ms[i], kt.launches[i]) for i, name in enumerate(KERNEL_CLASSES)}

    def adjoint_enable(self, on=True):
        """Keep each step's input so that step_adjoint can differentiate it."""
        _check(load().harmrad_adjoint_enable(self._h, 1 if on else 0), "adjoint_enable")

    def branch_signature(self, on=True):
        """Start (zeroed) or stop the per-cell branch signature of later steps."""
        _check(load().harmrad_branch_signature(self._h, 1 if on else 0), "branch_signature")

    def get_branch_signature(self):
        """The signature words of every cell (ghost-inclusive, uint64, numpy)."""
        ng = [4 if x > 1 else 0 for x in self.cfg["n"]]
        n = int(np.prod([self.cfg["n"][i] + 2 * ng[i] for i in range(3)]))
        out = np.empty(n, dtype=np.uint64)
        _check(load().harmrad_get_branch_signature(self._h, out.ctypes.data_as(ctypes.c_void_p), 0),
               "get_branch_signature")
        return out

    def adjoint_set_input(self, P, dt):
        """Record P (float64 CUDA tensor, active layout) and dt as the input of
        the step that the next step_adjoint differentiates (no step is run)."""
        P = P.contiguous()
        _check(load().harmrad_adjoint_set_input(self._h, ctypes.c_void_p(P.data_ptr()), float(dt), 1),
               "adjoint_set_input")

    def step_adjoint(self, gP_out):
        """Reverse-mode derivative of the last step: dL/dP^{n+1} -> (dL/dP^n,
        dL/dkappa_scale), time step fixed.  Torch CUDA tensors stay on the
        device; numpy arrays are copied through the host."""
        import torch
        gk = ctypes.c_double()
        if isinstance(gP_out, torch.Tensor):
            assert gP_out.is_cuda and gP_out.dtype == torch.float64
            gin = gP_out.contiguous()
            out = torch.empty_like(gin)
            _check(load().harmrad_step_adjoint(self._h, ctypes.c_void_p(gin.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), ctypes.byref(gk), 1),
                   "step_adjoint")
            return out, gk.value
        gin = np.ascontiguousarray(gP_out, dtype=np.float64)
        out = np.empty_like(gin)
        _check(load().harmrad_step_adjoint(self._h, gin.ctypes.data_as(ctypes.c_void_p),
                                           out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(gk), 0),
               "step_adjoint")
        return out, gk.value

    def autotune(self, reps=2):
        """Pick the fastest launch shapes on the current state (state kept)."""
        t = Tuning()
        _check(load().harmrad_autotune(self._h, int(reps), ctypes.byref(t)), "autotune")
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def tuning(self):
        t = Tuning()
        _check(load().harmrad_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        t = Tuning()
        _check(load().harmrad_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        for k, v in kw.items():
            setattr(t, k, v)
        _check(load().harmrad_set_tuning(self._h, ctypes.byref(t)), "set_tuning")

    def stats(self):
        s = Stats()
        _check(load().harmrad_get_stats(self._h, ctypes.byref(s)), "get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def status(self):
        st = np.empty(self.shape[1:], dtype=np.uint8)
        _check(load().harmrad_get_status(self._h, st.ctypes.data_as(ctypes.c_void_p), 0), "get_status")
        return st

    def iters(self):
        it = np.empty(self.shape[1:], dtype=np.int32)
        _check(load().harmrad_get_iters(self._h, it.ctypes.data_as(ctypes.c_void_p), 0), "get_iters")
        return it

    def fluxes(self, d):
        m = list(self.n)
        m[d - 1] += 1
        F = np.empty((NPRIM, m[2], m[1], m[0]))
        _check(load().harmrad_compute_fluxes(self._h, int(d), F.ctypes.data_as(ctypes.c_void_p)),
               "compute_fluxes")
        return F


class Batch(Grid):
    """A batch of independent grids ("boxes") in one context: every kernel of
    a step covers all boxes.  Per-box arrays are passed and returned as lists
    in box order; the context holds them concatenated."""

    def __init__(self, cfgs, precision=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise HarmradError("a CUDA device is required")
        L = load()
        self.cfgs = [dict(c) for c in cfgs]
        self.cfg = self.cfgs[0]
        arr = (Params * len(cfgs))(*[make_params(c, precision) for c in cfgs])
        self.params = arr
        self.shapes = [(NPRIM, c["n"][2], c["n"][1], c["n"][0]) for c in cfgs]
        self.sizes = [int(np.prod(s[1:])) for s in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.nact = int(self.offsets[-1])
        self.shape = (NPRIM * self.nact,)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(L.harmrad_init_batch(arr, len(cfgs), _stream_ptr(self.stream), ctypes.byref(h)),
               "harmrad_init_batch")
        self._h = h

    def pack(self, Ps):
        """List of [12,n3,n2,n1] arrays -> the context's flat layout (numpy)."""
        return np.concatenate([np.ascontiguousarray(P, dtype=np.float64).reshape(-1) for P in Ps])

    def unpack(self, flat, nv=NPRIM):
        out = []
        for b, s in enumerate(self.shapes):
            o, m = self.offsets[b], self.sizes[b]
            out.append(flat[nv * o:nv * (o + m)].reshape((nv,) + s[1:]) if nv > 1 else
                       flat[o:o + m].reshape(s[1:]))
        return out

    def set_prims(self, Ps):
        import torch
        if isinstance(Ps, torch.Tensor):
            assert Ps.is_cuda and Ps.dtype == torch.float64 and Ps.numel() == NPRIM * self.nact
            Ps = Ps.contiguous()
            _check(load().harmrad_set_prims(self._h, ctypes.c_void_p(Ps.data_ptr()), 1), "set_prims")
            return
        flat = self.pack(Ps)
        _check(load().harmrad_set_prims(self._h, flat.ctypes.data_as(ctypes.c_void_p), 0), "set_prims")

    def set_opacity_field(self, Ks):
        flat = np.concatenate([np.ascontiguousarray(K, dtype=np.float64).reshape(-1) for K in Ks])
        assert flat.size == self.nact
        _check(load().harmrad_set_opacity_field(self._h, flat.ctypes.data_as(ctypes.c_void_p), 0),
               "set_opacity_field")

    def get_prims(self, device=False):
        import torch
        if device:
            out = torch.empty(NPRIM * self.nact, dtype=torch.float64, device="cuda")
            _check(load().harmrad_get_prims(self._h, ctypes.c_void_p(out.data_ptr()), 1), "get_prims")
            return out
        out = np.empty(NPRIM * self.nact)
        _check(load().harmrad_get_prims(self._h, out.ctypes.data_as(ctypes.c_void_p), 0), "get_prims")
        return self.unpack(out)

    def status(self):
        st = np.empty(self.nact, dtype=np.uint8)
        _check(load().harmrad_get_status(self._h, st.ctypes.data_as(ctypes.c_void_p), 0), "get_status")
        return self.unpack(st, 1)

    def iters(self):
        it = np.empty(self.nact, dtype=np.int32)
        _check(load().harmrad_get_iters(self._h, it.ctypes.data_as(ctypes.c_void_p), 0), "get_iters")
        return self.unpack(it, 1)

    def fluxes(self, d):
        raise HarmradError("face fluxes are available for single-grid contexts only")


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def fp64_fma_rate(reps=5, stream=None):
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().harmrad_fp64_fma_rate(int(reps), ctypes.byref(t), _stream_ptr(stream)),
           "fp64_fma_rate")
    return t.value


def zone_physics(cfg, x, P):
    """Point-wise U, SM, F[3], speeds[3][4] at n points (numpy in, numpy out)."""
    import torch
    n = len(x)
    xd, Pd = _dev(x), _dev(P)
    U = torch.empty((n, 12), dtype=torch.float64, device="cuda")
    SM = torch.empty((n, 12), dtype=torch.float64, device="cuda")
    F = torch.empty((n, 3, 12), dtype=torch.float64, device="cuda")
    S = torch.empty((n, 3, 4), dtype=torch.float64, device="cuda")
    p = make_params(cfg)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(load().harmrad_zone_physics(ctypes.byref(p), n, vp(xd), vp(Pd), vp(U), vp(SM), vp(F), vp(S),
                                       _stream_ptr(None)), "zone_physics")
    return U.cpu().numpy(), SM.cpu().numpy(), F.cpu().numpy(), S.cpu().numpy()


def zone_implicit(cfg, x, Ustar, Ps, h, Sstar=None):
    """Implicit four-force solve of n independent zones (numpy in, numpy out).
    Sstar (n values of sqrt(-g) S u^t after the explicit update) adds the
    entropy equation to the back-up equations (harmrad_zone_implicit_full)."""
    import torch
    n = len(x)
    xd, Ud, Pd, hd = _dev(x), _dev(Ustar), _dev(Ps), _dev(np.broadcast_to(h, (n,)))
    Pout = torch.empty((n, 12), dtype=torch.float64, device="cuda")
    eT = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    meth = torch.empty(n, dtype=torch.uint8, device="cuda")
    p = make_params(cfg)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    if Sstar is None:
        _check(load().harmrad_zone_implicit(ctypes.byref(p), n, vp(xd), vp(Ud), vp(Pd), vp(hd), vp(Pout),
                                            vp(eT), vp(it), vp(meth), _stream_ptr(None)), "zone_implicit")
    else:
        Sd = _dev(np.broadcast_to(Sstar, (n,)))
        _check(load().harmrad_zone_implicit_full(ctypes.byref(p), n, vp(xd), vp(Ud), vp(Sd), vp(Pd), vp(hd),
                                                 vp(Pout), vp(eT), vp(it), vp(meth), _stream_ptr(None)),
               "zone_implicit_full")
    return Pout.cpu().numpy(), eT.cpu().numpy(), it.cpu().numpy(), meth.cpu().numpy()


def zone_method(cfg, x, Ustar, Ps, h, method, Sstar=None):
    """One Newton method alone on n zones (0 PMHD, 1 URAD, 2 PRAD, 3 staged
    PMHD, 4 staged URAD, 5 staged PRAD, 6/7/8 the entropy-based PMHD, URAD,
    PRAD, which need Sstar): (P[n][12], e_T[n], steps[n]) as numpy arrays."""
    import torch
    n = len(x)
    xd, Ud, Pd, hd = _dev(x), _dev(Ustar), _dev(Ps), _dev(np.broadcast_to(h, (n,)))
    Sd = _dev(np.broadcast_to(Sstar, (n,))) if Sstar is not None else None
    Pout = torch.empty((n, 12), dtype=torch.float64, device="cuda")
    eT = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    p = make_params(cfg)
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().harmrad_zone_method(ctypes.byref(p), n, vp(xd), vp(Ud), vp(Sd), vp(Pd), vp(hd), int(method),
                                      vp(Pout), vp(eT), vp(it), _stream_ptr(None)), "zone_method")
    return Pout.cpu().numpy(), eT.cpu().numpy(), it.cpu().numpy()
