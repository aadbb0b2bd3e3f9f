"""Seeded synthetic workloads for the HARMRAD step.

Each generator returns ``(cfg, P)``: a plain dict of run parameters (the
fields of ``harmrad_params``) and the initial primitives as a float64 array of
shape ``[12, n3, n2, n1]``.  The same bytes feed the CUDA library and the CPU
oracle.  Random draws use numpy's counter-based Philox generator with a fixed
key, so every run reproduces bit for bit on any host.

The workloads follow the shapes and value ranges the paper uses (McKinney et
al. 2014): a stiff uniform radiating box (Sec. 5 style relaxation), a
magnetised, radiation-supported torus on a Kerr-Schild grid with the paper's
spin a = 0.9375 and fiducial 256x128x64 resolution (Sec. 6), and periodic
Minkowski boxes with Gaussian radiation pulses (Sec. 5.3).  The torus builds
its divergence-free initial field from a vector potential and normalises it to
a plasma beta; those two set-up steps need sqrt(-g) and b^2 of a static
observer, which are written out below as closed forms of the Kerr-Schild
metric.  They are initial-condition formulas, not part of the time step.
"""
import math

import numpy as np

NP = 12
RHO, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3 = range(12)
PERIODIC, OUTFLOW, POLAR, COPY, FIXED = 0, 1, 2, 3, 4
PPM, MC = 0, 1
LAXF, HLL = 0, 1
OPAC_CONST, OPAC_KRAMERS, OPAC_FIELD = 0, 1, 2
RK3, IMEX2, IMEX2B, IMEX3 = 0, 1, 2, 3


def rng(seed):
    """Counter-based generator (Philox-4x64) keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


def base_params():
    return dict(
        n=[1, 1, 1], x0=[0.0, 0.0, 0.0], dx=[1.0, 1.0, 1.0],
        metric=0, a_spin=0.0, R0=0.0, hslope=0.3,
        bc=[PERIODIC] * 6,
        gam=5.0 / 3.0, a_rad=1.0, courant=0.5,
        opacity=OPAC_CONST, kappa_abs0=0.0, kappa_es0=0.0, kappa_scale=1.0, T_kappa_min=0.0,
        recon=PPM, flux=LAXF,
        gamma_rad_max=100.0, gamma_gas_max=50.0,
        floor_rho0=1e-10, floor_rho_pow=0.0, floor_u0=1e-12, floor_u_pow=0.0,
        bsq_rho_max=200.0, bsq_u_max=1e5, u_rho_max=1e10,
        newton_max=20, newton_tol=1e-12, integrator=0, implicit_eq=0, emf=0,
    )


def relax_box(n1=256, perturb=1e-4):
    """1D periodic Minkowski box, N=256: rho0=1, u_g=1e-2 (1 + A sin 2 pi x),
    Ebar = 2 a_rad T0^4 with a_rad T0^4 = u_g0, tau_abs = 10 per zone,
    kappa_es = 0.4.  Stiff relaxation toward radiative equilibrium."""
    cfg = base_params()
    dx = 1.0 / n1
    T0 = (cfg["gam"] - 1.0) * 1e-2
    a_rad = 1e-2 / T0 ** 4
    cfg.update(n=[n1, 1, 1], dx=[dx, 1.0, 1.0], a_rad=a_rad,
               opacity=OPAC_CONST, kappa_abs0=10.0 / dx, kappa_es0=0.4)
    x = (np.arange(n1) + 0.5) * dx
    P = np.zeros((NP, 1, 1, n1))
    P[RHO] = 1.0
    P[UU] = 1e-2 * (1.0 + perturb * np.sin(2 * np.pi * x))
    P[ER] = 2.0 * a_rad * T0 ** 4
    return cfg, P


# --- Kerr-Schild torus ---------------------------------------------------------

def _ks_setup(n, a=0.9375, hslope=0.3, rin=1.2, rout=50.0):
    cfg = base_params()
    x1a, x1b = math.log(rin), math.log(rout)
    cfg.update(n=list(n), x0=[x1a, 0.0, 0.0],
               dx=[(x1b - x1a) / n[0], 1.0 / n[1], 1.0 / n[2]],
               metric=1, a_spin=a, R0=0.0, hslope=hslope,
               bc=[OUTFLOW, OUTFLOW, POLAR, POLAR, PERIODIC, PERIODIC])
    return cfg


def _theta(x2, h):
    return np.pi * x2 + 0.5 * (1.0 - h) * np.sin(2 * np.pi * x2)


def _gaussian_torus(r, th):
    return np.exp(-((r - 15.0) / 4.0) ** 2 - (np.cos(th) / 0.3) ** 2)


def torus(n=(64, 32, 16), seed=12345, b_background=0.0, faces=False):
    """Seeded Kerr-Schild torus, a = 0.9375, r in [1.2, 50] log-spaced,
    theta concentrated toward the equator (h = 0.3):
    rho = max(G(r, theta) (1 + 0.02 sin phi_k), 1e-6 r^-1.5) with G a Gaussian
    in (r - 15, cos theta) and phi_k a random phase per zone;
    u_g = 0.01 rho^(4/3); gas and radiation at rest in the ZAMO frame;
    radiation in LTE (Ebar = a_rad T^4) with p_rad = p_gas at the density
    maximum; Kramers absorption (tau_abs = 10 per zone at the maximum) plus
    electron scattering; B from A_phi ~ max(rho - 0.2, 0) scaled so that
    max p_gas / max p_mag = 100.  b_background > 0 adds the field of
    A_phi = b_background (r sin theta)^2 (a weak vertical field threading the
    whole grid).  faces=True also returns the staggered field of the same
    potential, sqrt(-g) B^d on the d-faces as (x-faces [n3, n2, n1+1],
    y-faces [n3, n2+1, n1], z-faces [n3+1, n2, n1]): sqrt(-g) B^1 =
    d A_phi / dx2 and sqrt(-g) B^2 = -d A_phi / dx1 by differences of the
    corner values along the face, whose two-face averages are the
    cell-centred B."""
    cfg = _ks_setup(n)
    n1, n2, n3 = n
    a, h = cfg["a_spin"], cfg["hslope"]
    gam = cfg["gam"]
    x1c = cfg["x0"][0] + (np.arange(n1) + 0.5) * cfg["dx"][0]
    x2c = (np.arange(n2) + 0.5) * cfg["dx"][1]
    x1f = cfg["x0"][0] + np.arange(n1 + 1) * cfg["dx"][0]
    x2f = np.arange(n2 + 1) * cfg["dx"][1]
    r = np.exp(x1c)[None, None, :]
    th = _theta(x2c, h)[None, :, None]
    phase = rng(seed).uniform(0.0, 2 * np.pi, size=(n3, n2, n1))
    rho = np.maximum(_gaussian_torus(r, th) * (1.0 + 0.02 * np.sin(phase)), 1e-6 * r ** -1.5)
    ug = 0.01 * rho ** (4.0 / 3.0)
    T0 = (gam - 1.0) * 0.01
    a_rad = 3.0 / T0 ** 3  # a T0^4 / 3 = p_gas at rho = 1
    T = (gam - 1.0) * ug / rho
    # vector potential at cell corners (axisymmetric, unperturbed density)
    rf = np.exp(x1f)[None, :]
    thf = _theta(x2f, h)[:, None]
    A = np.maximum(_gaussian_torus(rf, thf) - 0.2, 0.0)  # [n2+1, n1+1]
    # static-observer metric pieces at cell centres (closed forms of Kerr-Schild)
    r2 = np.exp(x1c)[None, :]
    th2 = _theta(x2c, h)[:, None]
    Sig = r2 ** 2 + a * a * np.cos(th2) ** 2
    drdx1 = r2
    dthdx2 = np.pi * (1.0 + (1.0 - h) * np.cos(2 * np.pi * x2c))[:, None]
    gdet = Sig * np.abs(np.sin(th2)) * drdx1 * dthdx2 * 2 * np.pi
    B1c = (A[1:, :-1] + A[1:, 1:] - A[:-1, :-1] - A[:-1, 1:]) / (2 * cfg["dx"][1] * gdet)
    B2c = -(A[:-1, 1:] + A[1:, 1:] - A[:-1, :-1] - A[1:, :-1]) / (2 * cfg["dx"][0] * gdet)
    alpha2 = 1.0 / (1.0 + 2 * r2 / Sig)
    g11 = (1.0 + 2 * r2 / Sig) * drdx1 ** 2
    g22 = Sig * dthdx2 ** 2
    bsq = alpha2 * (g11 * B1c ** 2 + g22 * B2c ** 2)
    pg = (gam - 1.0) * ug
    pb_max = 0.5 * bsq.max()
    scale = math.sqrt(pg.max() / (100.0 * pb_max)) if pb_max > 0 else 0.0
    P = np.zeros((NP, n3, n2, n1))
    P[RHO] = rho
    P[UU] = ug
    Atot = scale * A
    if b_background > 0.0:
        Ab = b_background * (rf * np.sin(thf)) ** 2
        B1c = scale * B1c + (Ab[1:, :-1] + Ab[1:, 1:] - Ab[:-1, :-1] - Ab[:-1, 1:]) / (2 * cfg["dx"][1] * gdet)
        B2c = scale * B2c - (Ab[:-1, 1:] + Ab[1:, 1:] - Ab[:-1, :-1] - Ab[1:, :-1]) / (2 * cfg["dx"][0] * gdet)
        Atot = Atot + Ab
        scale = 1.0
    P[B1] = (scale * B1c)[None, :, :]
    P[B2] = (scale * B2c)[None, :, :]
    P[ER] = a_rad * T ** 4
    dx1 = cfg["dx"][0]
    kK = 10.0 * T0 ** 3.5 / (15.0 * dx1)
    cfg.update(a_rad=a_rad, opacity=OPAC_KRAMERS, kappa_abs0=kK, kappa_es0=0.4,
               T_kappa_min=1e-3 * T0,
               floor_rho0=1e-6, floor_rho_pow=-1.5, floor_u0=1e-8, floor_u_pow=-2.5)
    if faces:
        f1 = (Atot[1:, :] - Atot[:-1, :]) / cfg["dx"][1]           # [n2, n1+1]
        f2 = -(Atot[:, 1:] - Atot[:, :-1]) / cfg["dx"][0]          # [n2+1, n1]
        Bf = (np.broadcast_to(f1, (n3, n2, n1 + 1)).copy(), np.broadcast_to(f2, (n3, n2 + 1, n1)).copy(),
              np.zeros((n3 + 1, n2, n1)))
        return cfg, P, Bf
    return cfg, P


def generic_torus(n=(32, 16, 8), seed=12345):
    """The torus made differentiable in every zone, for derivative checks:
    a weak vertical background field (no zone with B = 0), velocity noise of
    amplitude 1e-4 in every gas and radiation component (no zone at rest, so
    no limiter sits on its kink at zero slope), field noise of relative size
    1e-3 in every component (no direction along which the field is constant;
    this noise is not divergence-free, which the step, constrained transport
    included, does not need), and an atmosphere three times above the floors
    (no floor acts on the initial state)."""
    cfg, P = torus(n, seed, b_background=1e-5)
    g = rng(seed + 1)
    P[U1:U3 + 1] += 1e-4 * g.standard_normal(P[U1:U3 + 1].shape)
    P[UR1:UR3 + 1] += 1e-4 * g.standard_normal(P[UR1:UR3 + 1].shape)
    bmag = np.sqrt(P[B1] ** 2 + P[B2] ** 2)
    P[B1] *= 1.0 + 1e-3 * g.standard_normal(bmag.shape)
    P[B2] *= 1.0 + 1e-3 * g.standard_normal(bmag.shape)
    P[B3] = 1e-3 * bmag * g.standard_normal(bmag.shape)
    r = np.exp(cfg["x0"][0] + (np.arange(n[0]) + 0.5) * cfg["dx"][0])[None, None, :]
    P[RHO] = np.maximum(P[RHO], 3.0 * cfg["floor_rho0"] * r ** cfg["floor_rho_pow"])
    P[UU] = np.maximum(P[UU], 3.0 * cfg["floor_u0"] * r ** cfg["floor_u_pow"])
    return cfg, P


def ks_random_state(n=(32, 16, 8), seed=9, recon=PPM, tau=10.0):
    """A random state on the Kerr-Schild grid of the torus (r in [1.2, 50],
    polar and outflow boundaries), for derivative checks: rho log-normal
    (sigma 0.5), u_g = 0.01 rho (1 +- 0.2), random velocities of ~0.1, field
    of ~0.02 and radiation-frame velocities of ~0.05 (orthonormal sizes),
    Ebar between 1 and 2 times a_rad T^4, Kramers absorption with optical
    depth ~tau per zone.  Zone-to-zone variations of order one keep every
    slope limiter away from its switching points for small perturbations."""
    cfg = _ks_setup(n)
    n1, n2, n3 = n
    gam = cfg["gam"]
    T0 = (gam - 1.0) * 0.01
    cfg.update(recon=recon, a_rad=1e-2 / T0 ** 4, opacity=OPAC_KRAMERS,
               kappa_abs0=tau * T0 ** 3.5 / cfg["dx"][0], kappa_es0=0.4, T_kappa_min=1e-3 * T0,
               floor_rho0=1e-12, floor_u0=1e-14, floor_rho_pow=0.0, floor_u_pow=0.0)
    g = rng(seed)
    shape = (n3, n2, n1)
    x1 = cfg["x0"][0] + (np.arange(n1) + 0.5) * cfg["dx"][0]
    x2 = (np.arange(n2) + 0.5) * cfg["dx"][1]
    r = np.exp(x1)[None, None, :]
    th = _theta(x2, cfg["hslope"])[None, :, None]
    P = np.zeros((NP,) + shape)
    P[RHO] = np.exp(0.5 * g.standard_normal(shape))
    P[UU] = 0.01 * P[RHO] * (1.0 + 0.2 * g.uniform(-1, 1, shape))
    # coordinate components of orthonormal sizes (dr/dx1 = r, r dtheta ~ pi r, r sin dphi = 2 pi r sin)
    sc = [1.0 / r, 1.0 / (np.pi * r) + 0.0 * th, 1.0 / (2 * np.pi * r * np.sin(th))]
    for c in range(3):
        P[U1 + c] = 0.1 * g.standard_normal(shape) * sc[c]
        P[B1 + c] = 0.02 * g.standard_normal(shape) * sc[c]
        P[UR1 + c] = 0.05 * g.standard_normal(shape) * sc[c]
    T = (gam - 1.0) * P[UU] / P[RHO]
    P[ER] = cfg["a_rad"] * T ** 4 * (1.0 + g.uniform(0, 1, shape))
    return cfg, P


# --- Minkowski boxes -------------------------------------------------------------

def minkowski_box(n=(16, 16, 16), seed=7, B_amp=0.05, vmax=0.3, kappa=(1e-2, 1e2),
                  recon=PPM, flux=LAXF):
    """Periodic 3D Minkowski box with random smooth-ish gas, field and
    radiation: rho log-normal (sigma 0.5), u_g = 0.01 rho (1 + noise),
    random velocities up to vmax, a random field of amplitude B_amp, a
    Gaussian radiation pulse, and a constant per-density absorption opacity
    (kappa_abs per length = kappa_abs0 * rho)."""
    cfg = base_params()
    n1, n2, n3 = n
    cfg.update(n=list(n), dx=[1.0 / n1, 1.0 / n2, 1.0 / n3], recon=recon, flux=flux)
    g = rng(seed)
    shape = (n3, n2, n1)
    P = np.zeros((NP,) + shape)
    P[RHO] = np.exp(0.5 * g.standard_normal(shape))
    P[UU] = 0.01 * P[RHO] * (1.0 + 0.2 * g.uniform(-1, 1, shape))
    v = g.standard_normal((3,) + shape)
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    speed = g.uniform(0.0, vmax, shape)
    gamma = 1.0 / np.sqrt(1.0 - speed ** 2)
    P[U1:U3 + 1] = v * (gamma * speed)[None]
    P[B1:B3 + 1] = B_amp * g.uniform(-1, 1, (3,) + shape)
    T = (cfg["gam"] - 1.0) * P[UU] / P[RHO]
    cfg["a_rad"] = 1e-2 / ((cfg["gam"] - 1.0) * 1e-2) ** 4
    zc = [(np.arange(m) + 0.5) / m - 0.5 for m in n]
    R2 = zc[2][:, None, None] ** 2 + zc[1][None, :, None] ** 2 + zc[0][None, None, :] ** 2
    P[ER] = cfg["a_rad"] * T ** 4 * (1.0 + 10.0 * np.exp(-R2 / 0.1 ** 2))
    ur = g.standard_normal((3,) + shape) * 0.05
    P[UR1:UR3 + 1] = ur
    kap = math.exp(g.uniform(math.log(kappa[0]), math.log(kappa[1])))
    cfg.update(opacity=OPAC_CONST, kappa_abs0=kap, kappa_es0=0.4 * kap / 10.0)
    return cfg, P


def box_batch(count=48, seed=4242, edge=(32, 128), tau=(1e-4, 1e6), vmax=0.3):
    """``count`` independent periodic 3D Minkowski unit boxes of uneven size,
    for one batched context.  Each edge is round(lo * (hi/lo)^U), U uniform,
    so sizes are log-uniform between edge[0] and edge[1] per direction.  Per
    box: rho log-normal (sigma 1), u_g = 0.01 rho, velocities of random
    direction and speed uniform up to vmax, B = 0, a Gaussian radiation pulse
    a T0^4 (1 + 100 exp(-r^2/w^2)), w = 0.1 of the box, T0 the mean gas temperature,
    radiation frame at rest in the ZAMO frame, and a per-zone absorption
    field whose optical depth per cell is log-uniform over ``tau`` (so Newton
    iteration counts are heavy-tailed), electron scattering kappa_es = 0.4.
    Returns (cfgs, Ps, Ks): per-box parameter dicts, primitives [12,n3,n2,n1]
    and absorption fields K [n3,n2,n1] (kappa_abs per length = K)."""
    g = rng(seed)
    lo, hi = edge
    cfgs, Ps, Ks = [], [], []
    gam = 5.0 / 3.0
    T0 = (gam - 1.0) * 1e-2
    for b in range(count):
        n = [int(round(lo * (hi / lo) ** g.uniform())) for _ in range(3)]
        n1, n2, n3 = n
        cfg = base_params()
        cfg.update(n=n, dx=[1.0 / n1, 1.0 / n2, 1.0 / n3], gam=gam, a_rad=1e-2 / T0 ** 4,
                   opacity=OPAC_FIELD, kappa_abs0=0.0, kappa_es0=0.4, kappa_scale=1.0)
        shape = (n3, n2, n1)
        P = np.zeros((NP,) + shape)
        P[RHO] = np.exp(g.standard_normal(shape))
        P[UU] = 0.01 * P[RHO]
        v = g.standard_normal((3,) + shape)
        v /= np.linalg.norm(v, axis=0, keepdims=True)
        speed = g.uniform(0.0, vmax, shape)
        P[U1:U3 + 1] = v * (speed / np.sqrt(1.0 - speed ** 2))[None]
        zc = [(np.arange(m) + 0.5) / m - 0.5 for m in n]
        R2 = zc[2][:, None, None] ** 2 + zc[1][None, :, None] ** 2 + zc[0][None, None, :] ** 2
        P[ER] = cfg["a_rad"] * T0 ** 4 * (1.0 + 100.0 * np.exp(-R2 / 0.1 ** 2))
        dxm = min(cfg["dx"])
        K = np.exp(g.uniform(math.log(tau[0]), math.log(tau[1]), shape)) / dxm
        cfgs.append(cfg)
        Ps.append(P)
        Ks.append(K)
    return cfgs, Ps, Ks


def linear_wave(N, bg, mode):
    """1D periodic Minkowski box [0, 1) of N zones carrying one linear
    eigenmode q = Re[q_a + dq exp(-i k x)] at t = 0 (Sec. 5 linear waves): bg
    holds rho, e_gas, gam, k; mode holds tau (kappa_es), P (p_rad/p_gas), B0
    and the complex amplitudes [re, im] drho, dug, dux, duy, dBy, dE, dFx,
    dFy (fluid-frame radiation energy and flux).  To first order the
    radiation-frame energy density equals the fluid-frame one and the
    radiation frame moves relative to the fluid with v = 3 F / (4 E), so
    u~_rad = u~ + 3 dF / (4 E_a).  The opacity tau is absorption, with the
    background radiation in equilibrium with the gas (a_rad T^4 = E_a,
    T = p/rho) and no scattering: the printed eigenvalues are those of the
    linearised equations with absorption (the accompanying text names the
    opacity scattering; with scattering alone no mode has these
    eigenvalues)."""
    cfg = base_params()
    gam = bg["gam"]
    pg = (gam - 1.0) * bg["e_gas"]
    Ea = 3.0 * mode["P"] * pg
    T0 = pg / bg["rho"]
    cfg.update(n=[N, 1, 1], dx=[1.0 / N, 1.0, 1.0], gam=gam, a_rad=Ea / T0 ** 4, opacity=OPAC_CONST,
               kappa_abs0=mode["tau"], kappa_es0=0.0, recon=PPM, flux=LAXF,
               floor_rho0=1e-12, floor_u0=1e-14)
    x = (np.arange(N) + 0.5) / N
    ph = np.exp(-1j * bg["k"] * x)

    def pert(key):
        re, im = mode[key]
        return np.real((re + 1j * im) * ph)

    P = np.zeros((NP, 1, 1, N))
    P[RHO] = bg["rho"] + pert("drho")
    P[UU] = bg["e_gas"] + pert("dug")
    P[U1] = pert("dux")
    P[U2] = pert("duy")
    P[B1] = mode["B0"]
    P[B2] = mode["B0"] + pert("dBy")
    P[ER] = Ea + pert("dE")
    P[UR1] = P[U1] + 0.75 * pert("dFx") / Ea
    P[UR2] = P[U2] + 0.75 * pert("dFy") / Ea
    return cfg, P


def wave_amplitude(rho, k):
    """Complex amplitude of the exp(-i k x) mode of rho on [0, 1)."""
    N = rho.size
    x = (np.arange(N) + 0.5) / N
    return 2.0 / N * np.sum((rho.ravel() - rho.mean()) * np.exp(1j * k * x))


def thin_pulse(n=(50, 50, 50), L=100.0, w=5.0, T_a=1e6, a_rad=8.77e-12):
    """Optically thin 3D radiation pulse (Sec. 5, 3D Cartesian Minkowski):
    kappa = 0, rho0 = 1, gas temperature T_a, radiation temperature
    T_a (1 + 100 exp(-r^2/w^2)), Ebar = a_rad T_rad^4, centred in a periodic
    box [-L/2, L/2)^3 of n zones per side.  Temperatures are in code units of
    m_b c^2/k_b; a_rad = 8.77e-12 in these units as the paper gives it."""
    cfg = base_params()
    n1, n2, n3 = n
    cfg.update(n=list(n), x0=[-L / 2] * 3, dx=[L / n1, L / n2, L / n3],
               opacity=OPAC_CONST, kappa_abs0=0.0, kappa_es0=0.0)
    Tg = T_a / 1.0888e13  # K -> m_b c^2 / k_b
    cfg["a_rad"] = a_rad
    zc = [cfg["x0"][i] + (np.arange(m) + 0.5) * cfg["dx"][i] for i, m in enumerate(n)]
    R2 = zc[2][:, None, None] ** 2 + zc[1][None, :, None] ** 2 + zc[0][None, None, :] ** 2
    P = np.zeros((NP, n3, n2, n1))
    P[RHO] = 1.0
    P[UU] = Tg / (cfg["gam"] - 1.0)
    Trad = Tg * (1.0 + 100.0 * np.exp(-R2 / w ** 2))
    P[ER] = cfg["a_rad"] * Trad ** 4
    return cfg, P


def thick_pulse(n1=100, L=100.0, w=5.0, kappa_es=1e3, T_a=1e6, a_rad=8.77e-12):
    """Optically thick planar radiation pulse (Sec. 5, 1D): radiation
    temperature T_a (1 + 100 exp(-x^2/w^2)) on n1 zones over [-L/2, L/2)
    (periodic), scattering opacity kappa_es per unit length at rho0 = 1, no
    absorption, gas at rest at temperature T_a (K, converted to m_b c^2 / k_b),
    a_rad = 8.77e-12 in these units (the paper's value).  The radiation energy is
    25 orders below the gas energy, so it diffuses as a test field with
    D = 1/(3 kappa_es)."""
    cfg = base_params()
    cfg.update(n=[n1, 1, 1], x0=[-L / 2, 0.0, 0.0], dx=[L / n1, 1.0, 1.0],
               opacity=OPAC_CONST, kappa_abs0=0.0, kappa_es0=kappa_es, a_rad=a_rad)
    Tg = T_a / 1.0888e13
    x = cfg["x0"][0] + (np.arange(n1) + 0.5) * cfg["dx"][0]
    P = np.zeros((NP, 1, 1, n1))
    P[RHO] = 1.0
    P[UU] = Tg / (cfg["gam"] - 1.0)
    P[ER] = cfg["a_rad"] * (Tg * (1.0 + 100.0 * np.exp(-x ** 2 / w ** 2))) ** 4
    return cfg, P


def thick_pulse_exact(x, t, L=100.0, w=5.0, kappa_es=1e3, T_a=1e6, a_rad=8.77e-12, images=2):
    """Solution of dE/dt = D d2E/dx2, D = 1/(3 kappa_es), from the thick
    pulse's initial radiation energy: its binomial expansion
    a T^4 sum_m C(4,m) 100^m exp(-m x^2/w^2) is a sum of Gaussians that each
    spread on their own (periodic images included)."""
    D = 1.0 / (3.0 * kappa_es)
    Tg = T_a / 1.0888e13
    x = np.asarray(x, dtype=float)
    E = np.ones_like(x)
    for m in range(1, 5):
        t0 = w * w / (4.0 * m * D)
        s = np.zeros_like(x)
        for k in range(-images, images + 1):
            s += np.exp(-(x - k * L) ** 2 / (4.0 * D * (t + t0)))
        E += math.comb(4, m) * 100.0 ** m * math.sqrt(t0 / (t + t0)) * s
    return a_rad * Tg ** 4 * E


def shock_tube(state, n1=800, xlim=(-20.0, 20.0), recon=PPM, flux=LAXF):
    """1D radiative shock tube (Sec. 5, HD radiative shocks): the left and
    right states (rho0, p_g, u^x, Ehat) of ``state`` (keys L, R, gam, sigma,
    kappa) on either side of x = 0, LTE radiation moving with the gas (u~_rad
    = u~, Ebar = Ehat), a_rad = 4 sigma, absorption opacity kappa rho0, no
    scattering, zero-gradient ends with inflow allowed."""
    cfg = base_params()
    gam = float(state["gam"])
    x0, x1 = xlim
    dx = (x1 - x0) / n1
    cfg.update(n=[n1, 1, 1], x0=[x0, 0.0, 0.0], dx=[dx, 1.0, 1.0], gam=gam,
               a_rad=4.0 * float(state["sigma"]), opacity=OPAC_CONST, kappa_abs0=float(state["kappa"]),
               kappa_es0=0.0, recon=recon, flux=flux, bc=[COPY, COPY] + [PERIODIC] * 4,
               floor_rho0=1e-12, floor_u0=1e-14)
    x = x0 + (np.arange(n1) + 0.5) * dx
    P = np.zeros((NP, 1, 1, n1))
    for side, sel in (("L", x < 0.0), ("R", x >= 0.0)):
        rho, pg, ux, E = (float(v) for v in state[side])
        P[RHO][..., sel] = rho
        P[UU][..., sel] = pg / (gam - 1.0)
        P[U1][..., sel] = ux
        P[ER][..., sel] = E
        P[UR1][..., sel] = ux
    return cfg, P


# CGS constants for the static atmosphere's physical units
_G, _C, _MSUN = 6.67430e-8, 2.99792458e10, 1.98847e33
_MP, _KB, _ARAD = 1.67262192e-24, 1.380649e-16, 7.5657e-15


def _m1_from_flux(E, F):
    """Radiation-frame energy density and Lorentz factor of an M1 field with
    lab (observer-frame) energy density E and flux F along one axis:
    E = Ebar (4 g^2 - 1)/3, F = 4/3 Ebar g^2 v (Sec. 3, Eq. Rlab), so
    F/E = 4 g^2 v / (4 g^2 - 1), solved for g by bisection."""
    ratio = F / E
    lo, hi = 1.0, 1e4
    for _ in range(200):
        g = math.sqrt(lo * hi)
        v = math.sqrt(1.0 - 1.0 / (g * g))
        if 4 * g * g * v / (4 * g * g - 1) > ratio:
            hi = g
        else:
            lo = g
    g = math.sqrt(lo * hi)
    return E * 3.0 / (4 * g * g - 1), g


def static_atmosphere(f, n1=40, r_in=1e6, r_out=1.4e6, rho_in_cgs=1e-15, T_in_K=1e6, flux_ratio=0.99999):
    """The static radiative atmosphere of the paper's Sec. 5 ("Static
    Radiative Atmosphere in 1D Spherical Polar Minkowski"): a polytropic
    atmosphere p = K rho0^Gamma on a Schwarzschild grid (Kerr-Schild, a = 0)
    from r = 1e6 to 1.4e6, one equatorial theta cell (0.99 to 1.01 pi/2), held
    up by gravity, its pressure gradient and the radiation force of a flux
    F = F_in (r_in/r)^2 with F_in = f F_Edd, F_Edd = 1/(kappa_es r_in^2);
    scattering only (kappa_abs = 0, kappa_es = 0.4 cm^2/g), M = 1 solar mass,
    rho0 = 1e-15 g/cm^3 and T = 1e6 K at r_in, E = F/0.99999.  Both radial
    boundaries are fixed at the analytic state (Eqs. rho, f); velocities start
    at zero.  The radial cells are uniform in ln r (the grid's map), not in r.
    The gas is fully ionised hydrogen (mean molecular weight 1/2, so
    p = 2 rho0 k T / m_p): with weight 1 the analytic atmospheres of the two
    lowest luminosities would end inside the grid (rho0 -> 0 at r = 1.30e6
    and 1.34e6), which the paper's runs cannot have done.

    Returns (cfg, P, info): P holds every cell including the 4 ghosts per
    radial side ([12, 1, 1, n1 + 8], for harmrad_set_prims_ghosts); info the
    cell radii, the analytic density and ZAMO-frame radial flux, and the unit
    conversions."""
    cfg = base_params()
    L = _G * _MSUN / _C ** 2                      # length unit GM/c^2
    rho_u = _MSUN / L ** 3                        # density unit
    T_u = _MP * _C ** 2 / _KB                     # temperature unit m_p c^2 / k_B
    kes = 0.4 * rho_u * L                         # kappa_es per length per unit density
    a_rad = _ARAD * T_u ** 4 / (rho_u * _C ** 2)
    gam = 5.0 / 3.0
    rho_in, T_in = rho_in_cgs / rho_u, 2.0 * T_in_K / T_u   # p/rho0 = 2 k T / (m_p c^2)
    K = rho_in * T_in / rho_in ** gam             # p = rho0 T at r_in
    x1a, x1b = math.log(r_in), math.log(r_out)
    dx1 = (x1b - x1a) / n1
    cfg.update(n=[n1, 1, 1], x0=[x1a, 0.495, 0.0], dx=[dx1, 0.01, 1.0], metric=1, a_spin=0.0, R0=0.0,
               hslope=1.0, bc=[FIXED, FIXED, PERIODIC, PERIODIC, PERIODIC, PERIODIC], gam=gam,
               a_rad=a_rad, opacity=OPAC_CONST, kappa_abs0=0.0, kappa_es0=kes, gamma_rad_max=200.0,
               floor_rho0=1e-60, floor_u0=1e-70)
    F_edd = 1.0 / (kes * r_in ** 2)
    C = gam * K / (gam - 1.0) * rho_in ** (gam - 1.0) - (1.0 - f) / r_in
    ng = 4
    ii = np.arange(-ng, n1 + ng)
    r = np.exp(x1a + (ii + 0.5) * dx1)
    rho = ((gam - 1.0) / (gam * K) * (C + (1.0 - f) / r)) ** (1.0 / (gam - 1.0))
    Fz = f * F_edd * (r_in / r) ** 2
    P = np.zeros((NP, 1, 1, len(ii)))
    P[RHO, 0, 0] = rho
    P[UU, 0, 0] = K * rho ** gam / (gam - 1.0)
    for m in range(len(ii)):
        Ez = Fz[m] / flux_ratio
        Ebar, g = _m1_from_flux(Ez, Fz[m])
        # u~^r in the internal chart: orthonormal g v over sqrt(g_{x1 x1}),
        # g_{x1 x1} = (1 + 2/r) r^2 for Kerr-Schild with a = 0 and r = e^x1
        P[ER, 0, 0, m] = Ebar
        P[UR1, 0, 0, m] = math.sqrt(g * g - 1.0) / math.sqrt((1.0 + 2.0 / r[m]) * r[m] ** 2)
    info = {"r": r, "rho": rho, "Fz": Fz, "F_edd": F_edd, "K": K, "kes": kes, "ng": ng,
            "units": {"length_cm": L, "density_gcc": rho_u, "temperature_K": T_u}}
    return cfg, P, info


def random_states(n, seed=3, metric=0, gamma_max=50.0, magnetised=True, gamma_rad_max=20.0):
    """Random point states for per-zone tests: positions x[n,4] (internal
    coordinates) and primitives P[n,12] spanning density, temperature,
    Lorentz factor (gas up to gamma_max, radiation frame up to gamma_rad_max)
    and radiation ranges, plus a parameter
    dict for the chosen metric (0 Minkowski, 1 Kerr-Schild a = 0.9375)."""
    g = rng(seed)
    cfg = base_params() if metric == 0 else _ks_setup((64, 32, 16))
    cfg.update(a_rad=1.0, opacity=OPAC_CONST, kappa_abs0=1.0, kappa_es0=0.4)
    x = np.zeros((n, 4))
    if metric == 0:
        x[:, 1:] = g.uniform(0, 1, (n, 3))
    else:
        x[:, 1] = np.log(g.uniform(1.2, 50.0, n))
        x[:, 2] = g.uniform(0.03, 0.97, n)
        x[:, 3] = g.uniform(0, 1, n)
    P = np.zeros((n, NP))
    P[:, RHO] = np.exp(g.uniform(np.log(1e-4), np.log(1e2), n))
    P[:, UU] = P[:, RHO] * np.exp(g.uniform(np.log(1e-5), np.log(10.0), n))
    lg = g.uniform(0.0, np.log(gamma_max), n)
    gam = np.exp(lg)
    d = g.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    P[:, U1:U3 + 1] = d * np.sqrt(gam ** 2 - 1.0)[:, None]
    if magnetised:
        P[:, B1:B3 + 1] = g.standard_normal((n, 3)) * np.sqrt(P[:, RHO])[:, None] * 0.3
    P[:, ER] = P[:, UU] * np.exp(g.uniform(np.log(1e-3), np.log(1e3), n))
    lgr = g.uniform(0.0, np.log(gamma_rad_max), n)
    gr = np.exp(lgr)
    d2 = g.standard_normal((n, 3))
    d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    P[:, UR1:UR3 + 1] = d2 * np.sqrt(gr ** 2 - 1.0)[:, None]
    if metric == 1:
        # coordinate components: scale by the local radius so that the
        # physical speeds stay in range (g_ii grows like r^2 in these charts)
        r = np.exp(x[:, 1])
        for c, s in ((U1, r), (U2, r * np.pi), (U3, r * 2 * np.pi)):
            P[:, c] /= s
            P[:, c + 7] /= s
        P[:, B1:B3 + 1] /= r[:, None] ** 2
    return cfg, x, P
