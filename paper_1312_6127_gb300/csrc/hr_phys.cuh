// Per-zone GRRMHD + M1 physics for sm_103a, evaluated in registers.
//
// Conventions follow Sec. 2-4 of McKinney et al. (2014): c = G = M = 1,
// Heaviside-Lorentz field, ZAMO-relative 4-velocities u~^i as primitives.
// Every function is templated on the metric (0 Minkowski Cartesian,
// 1 Kerr-Schild with the modified spherical-polar map) and, where the split
// precision path uses it, on the real type.  The metric is never streamed:
// each zone or face evaluates it from its internal coordinates.  Contractions
// are written for the sparsity of the Kerr-Schild metric in (t, r, theta, phi)
// charts: g_{t theta} = g_{r theta} = g_{theta phi} = 0 and g^{t phi} = 0.
#pragma once
#include <type_traits>

#include "hr_dual.cuh"
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace hr {

enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3, NPR = 12 };
enum { MINK = 0, KS = 1 };

// Physics and solver parameters shared by every grid of a context (kernel
// argument, read from the constant bank).
struct DevParams {
  int act[3];        // 1 if the direction is active (n > 1) in every grid
  int metric;
  double a, R0, h;
  int bc[6];
  double gam, a_rad, courant;
  int opacity;
  double kabs0, kes0, kscale, Tmin;
  int recon, flux;
  double grad_max, ggas_max, ymax_rad;
  double rf0, rfp, uf0, ufp, bsq_rho_max, bsq_u_max, u_rho_max;
  int newton_max;
  double newton_tol;
  int precision;
  int integrator;  // 0 RK3, 1 IMEX2, 2 IMEX2B, 3 IMEX3 (Sec. 4.1)
  int implicit_eq;  // 0 energy equations (entropy as back-up, RK3), 1 entropy in every zone
  int emf;          // 0 flux-CT, 1 staggered field with the 4-state upwind EMF
  // FP32 copies of the parameters the FP32 tangent pass reads (converted once
  // on the host, not per use on the device)
  float gm1f, ymaxf, Tminf, kabs0f, kes0f, aradf;
  // branch signature (a test instrument; null unless enabled): per cell a
  // 64-bit word into which every branch decision of the step is folded
  unsigned long long* sig;
  int sig_salt;  // sub-step of the decisions (0: the CFL pass)
};

// Fold one decision `code` of kernel `kernel` about cell `cell` (index into
// the context's cell arrays) into the branch signature.  Two runs took the
// same branches everywhere if and only if their words agree (up to 64-bit
// hash collisions).  The decision is hashed with the kernel and the sub-step,
// and words combine by XOR, so the order in which threads add them does not
// matter.
__device__ __forceinline__ unsigned long long sig_hash(unsigned long long a, unsigned long long b) {
  unsigned long long h = (a * 0x9E3779B97F4A7C15ULL) ^ (b + 0x632BE59BD9B4E019ULL);
  h ^= h >> 29;
  h *= 0xBF58476D1CE4E5B9ULL;
  h ^= h >> 32;
  h *= 0x94D049BB133111EBULL;
  h ^= h >> 31;
  return h;
}
__device__ __forceinline__ void sig_put(const DevParams& p, long long cell, unsigned kernel,
                                        unsigned long long code) {
  atomicXor(p.sig + cell, sig_hash(((unsigned long long)kernel << 32) | (unsigned)p.sig_salt, code));
}

// Geometry of one grid of a context: sizes, ghost depth, strides, internal
// coordinates, boundary conditions and the grid's offsets in the context's
// cell-indexed and active-zone-indexed arrays (one grid per box of a batch).
struct BoxGeo {
  int n[3], ng[3], N[3];
  long long ntot, nact;
  long long str[3];  // strides of the ghost-inclusive array per direction
  double x0[3], dx[3];
  int bc[6];
  long long coff;    // first cell of this grid in cell-indexed arrays
  long long aoff;    // first active zone of this grid in active-zone arrays
  long long goff;    // first double of this grid's metric table (-1: none)
};

// ----------------------------------------------------------------- geometry
template <int MET, typename R>
struct Geo {
  R g00, g01, g03, g11, g13, g22, g33;  // covariant, nonzero pattern of KS
  R G00, G01, G11, G13, G22, G33;       // contravariant
  R gdet, alpha, ialpha;

  __device__ __forceinline__ void lower(const R v[4], R w[4]) const {
    if constexpr (MET == MINK) {
      w[0] = -v[0];
      w[1] = v[1];
      w[2] = v[2];
      w[3] = v[3];
    } else {
      w[0] = g00 * v[0] + g01 * v[1] + g03 * v[3];
      w[1] = g01 * v[0] + g11 * v[1] + g13 * v[3];
      w[2] = g22 * v[2];
      w[3] = g03 * v[0] + g13 * v[1] + g33 * v[3];
    }
  }
  // g_ij v^i v^j over the spatial block
  __device__ __forceinline__ R sq3(R v1, R v2, R v3) const {
    if constexpr (MET == MINK) return v1 * v1 + v2 * v2 + v3 * v3;
    else return g11 * v1 * v1 + g22 * v2 * v2 + g33 * v3 * v3 + R(2) * g13 * v1 * v3;
  }
  // g^{t d}, g^{d d}, g_{d d} for d = 1..3
  __device__ __forceinline__ R Gt(int d) const {
    if constexpr (MET == MINK) return R(0);
    else return d == 1 ? G01 : R(0);
  }
  __device__ __forceinline__ R Gdd(int d) const {
    if constexpr (MET == MINK) return R(1);
    else return d == 1 ? G11 : (d == 2 ? G22 : G33);
  }
  __device__ __forceinline__ R gdd(int d) const {
    if constexpr (MET == MINK) return R(1);
    else return d == 1 ? g11 : (d == 2 ? g22 : g33);
  }
  __device__ __forceinline__ R Gtt() const {
    if constexpr (MET == MINK) return R(-1);
    else return G00;
  }
  // contravariant spatial components of a covariant 4-vector: g^{i mu} w_mu
  __device__ __forceinline__ void raise3(const R w[4], R v[3]) const {
    if constexpr (MET == MINK) {
      v[0] = w[1];
      v[1] = w[2];
      v[2] = w[3];
    } else {
      v[0] = G01 * w[0] + G11 * w[1] + G13 * w[3];
      v[1] = G22 * w[2];
      v[2] = G13 * w[1] + G33 * w[3];
    }
  }
  // g^{t mu} w_mu
  __device__ __forceinline__ R raise_t(const R w[4]) const {
    if constexpr (MET == MINK) return -w[0];
    else return G00 * w[0] + G01 * w[1];
  }
};

template <typename R> __device__ __forceinline__ R rsqrt_(R x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }

// Geometry of another scalar type (the adjoint evaluates the physics on dual
// numbers at the same, constant, metric).
template <typename T, int MET, typename R>
__device__ __forceinline__ Geo<MET, T> geo_cast(const Geo<MET, R>& a) {
  Geo<MET, T> g;
  g.g00 = T(a.g00); g.g01 = T(a.g01); g.g03 = T(a.g03); g.g11 = T(a.g11); g.g13 = T(a.g13);
  g.g22 = T(a.g22); g.g33 = T(a.g33);
  g.G00 = T(a.G00); g.G01 = T(a.G01); g.G11 = T(a.G11); g.G13 = T(a.G13); g.G22 = T(a.G22);
  g.G33 = T(a.G33);
  g.gdet = T(a.gdet); g.alpha = T(a.alpha); g.ialpha = T(a.ialpha);
  return g;
}

// Kerr-Schild metric in the internal chart at (x1, x2): covariant components
// scaled by the diagonal map Jacobian, the closed-form inverse of the
// Kerr-Schild metric (g^{tt} = -(1+2r/S), g^{tr} = 2r/S, g^{rr} = D/S,
// g^{r phi} = a/S, g^{theta theta} = 1/S, g^{phi phi} = 1/(S sin^2)),
// sqrt(-g) = S |sin theta| J1 J2 J3 and the lapse 1/sqrt(1 + 2r/S).
template <int MET, typename R>
__device__ __forceinline__ Geo<MET, R> make_geo(const DevParams& p, R x1, R x2) {
  Geo<MET, R> g;
  if constexpr (MET == MINK) {
    g.g00 = R(-1); g.g01 = R(0); g.g03 = R(0); g.g11 = R(1); g.g13 = R(0); g.g22 = R(1); g.g33 = R(1);
    g.G00 = R(-1); g.G01 = R(0); g.G11 = R(1); g.G13 = R(0); g.G22 = R(1); g.G33 = R(1);
    g.gdet = R(1);
    g.alpha = R(1);
    g.ialpha = R(1);
    (void)x1; (void)x2; (void)p;
  } else {
    const R a = R(p.a), hh = R(p.h);
    const R pi = R(3.14159265358979323846);
    R ex = exp(x1);
    R r = R(p.R0) + ex;
    R s2x, c2x;
    if constexpr (sizeof(R) == 8) sincospi(R(2) * x2, &s2x, &c2x);
    else sincospif(R(2) * x2, &s2x, &c2x);
    R th = pi * x2 + R(0.5) * (R(1) - hh) * s2x;
    R sth, cth;
    sincos(th, &sth, &cth);
    R J1 = ex, J2 = pi * (R(1) + (R(1) - hh) * c2x), J3 = R(2) * pi;
    R s2 = sth * sth;
    R S = r * r + a * a * cth * cth;
    R iS = R(1) / S;
    R tr = R(2) * r * iS;
    g.g00 = -(R(1) - tr);
    g.g01 = tr * J1;
    g.g03 = -a * tr * s2 * J3;
    g.g11 = (R(1) + tr) * J1 * J1;
    g.g13 = -a * s2 * (R(1) + tr) * J1 * J3;
    g.g22 = S * J2 * J2;
    g.g33 = s2 * (S + a * a * s2 * (R(1) + tr)) * J3 * J3;
    R D = r * r - R(2) * r + a * a;
    const R iJ1 = R(1) / J1, iJ2 = R(1) / J2, iJ3 = R(1.0 / (2.0 * 3.14159265358979323846));
    g.G00 = -(R(1) + tr);
    g.G01 = tr * iJ1;
    g.G11 = D * iS * iJ1 * iJ1;
    g.G13 = a * iS * iJ1 * iJ3;
    g.G22 = iS * iJ2 * iJ2;
    g.G33 = iS * iJ3 * iJ3 / s2;
    g.gdet = S * fabs(sth) * J1 * J2 * J3;
    g.alpha = rsqrt_<R>(R(1) + tr);
    g.ialpha = (R(1) + tr) * g.alpha;
  }
  return g;
}

// ------------------------------------------------------------- 4-vectors
// u^t = gamma/alpha, u^i = u~^i - gamma alpha g^{ti}, gamma^2 = 1 + g_ij u~^i u~^j.
// The same with the Lorentz factor gamma of (q1, q2, q3) already known.
template <int MET, typename R>
__device__ __forceinline__ void fourvel_g(const Geo<MET, R>& g, R q1, R q2, R q3, R gm, R ucon[4], R ucov[4]) {
  if constexpr (MET == MINK) {
    ucon[0] = gm;
    ucon[1] = q1;
    ucon[2] = q2;
    ucon[3] = q3;
  } else {
    ucon[0] = gm * g.ialpha;
    ucon[1] = q1 - gm * g.alpha * g.G01;
    ucon[2] = q2;
    ucon[3] = q3;
  }
  g.lower(ucon, ucov);
}

template <int MET, typename R>
__device__ __forceinline__ void fourvel(const Geo<MET, R>& g, R q1, R q2, R q3, R ucon[4],
                                        R ucov[4], R* gamma) {
  R gm = sqrt(R(1) + g.sq3(q1, q2, q3));
  *gamma = gm;
  if constexpr (MET == MINK) {
    ucon[0] = gm;
    ucon[1] = q1;
    ucon[2] = q2;
    ucon[3] = q3;
  } else {
    ucon[0] = gm * g.ialpha;
    ucon[1] = q1 - gm * g.alpha * g.G01;
    ucon[2] = q2;
    ucon[3] = q3;
  }
  g.lower(ucon, ucov);
}

// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t, b^2 = b^mu b_mu.
template <int MET, typename R>
__device__ __forceinline__ void bvec_iut(const Geo<MET, R>& g, const R ucon[4], const R ucov[4],
                                         R iut, R Bx, R By, R Bz, R bcon[4], R bcov[4], R* bsq) {
  R bt = Bx * ucov[1] + By * ucov[2] + Bz * ucov[3];
  bcon[0] = bt;
  bcon[1] = (Bx + bt * ucon[1]) * iut;
  bcon[2] = (By + bt * ucon[2]) * iut;
  bcon[3] = (Bz + bt * ucon[3]) * iut;
  g.lower(bcon, bcov);
  *bsq = bcon[0] * bcov[0] + bcon[1] * bcov[1] + bcon[2] * bcov[2] + bcon[3] * bcov[3];
}

template <int MET, typename R>
__device__ __forceinline__ void bvec(const Geo<MET, R>& g, const R ucon[4], const R ucov[4], R Bx,
                                     R By, R Bz, R bcon[4], R bcov[4], R* bsq) {
  bvec_iut<MET, R>(g, ucon, ucov, R(1) / ucon[0], Bx, By, Bz, bcon, bcov, bsq);
}

// Specific entropy of the gas (Sec. 2, Eq. S): s = log(p^n / rho0^(n+1)),
// n = 1/(Gamma - 1); the conserved entropy sqrt(-g) S u^t is sqrt(-g) rho0 u^t s.
template <typename R>
__device__ __forceinline__ R entropy_per_baryon(const DevParams& p, R rho, R ug) {
  if constexpr (std::is_same<R, double>::value) {
    // n = 3/2: p^n / rho^(n+1) = x sqrt(x) / rho with x = p / rho, one
    // logarithm (FP64 only: the product would leave FP32's range first)
    if (p.gam == 5.0 / 3.0) {
      const R ir = R(1) / rho;
      const R x = R(2.0 / 3.0) * ug * ir;
      return log(x * sqrt(x) * ir);
    }
  }
  const R n = R(1.0 / (p.gam - 1.0));
  return n * log(R(p.gam - 1.0) * ug) - (n + R(1)) * log(rho);
}

// Opacities per length at density rho and gas temperature T; kf is the
// zone's absorption opacity when the opacity is a per-zone field; ks the
// global opacity scale (kappa_scale; a separate argument so that the adjoint
// can differentiate with respect to it).
template <typename R>
__device__ __forceinline__ void opacity_ks(const DevParams& p, R rho, R T, R kf, R ks, R* kabs, R* ksca) {
  if (p.opacity == 2) {
    *kabs = ks * kf;
  } else if (p.opacity == 1) {
    R Tc = T > R(p.Tmin) ? T : R(p.Tmin);
    R T2 = Tc * Tc;
    R t35;
    if constexpr (!std::is_same<R, float>::value) {
      t35 = rsqrt_<R>(T2 * T2 * T2 * Tc);  // T^-3.5 = 1/sqrt(T^7): one reciprocal square root
    } else {
      t35 = rsqrt_<R>(Tc) / (T2 * Tc);  // T^7 would underflow in FP32
    }
    *kabs = ks * R(p.kabs0) * rho * rho * t35;
  } else {
    *kabs = ks * R(p.kabs0) * rho;
  }
  *ksca = ks * R(p.kes0) * rho;
}

template <typename R>
__device__ __forceinline__ void opacity_T(const DevParams& p, R rho, R T, R kf, R* kabs, R* ksca) {
  opacity_ks<R>(p, rho, T, kf, R(p.kscale), kabs, ksca);
}

template <typename R>
__device__ __forceinline__ void opacity(const DevParams& p, R rho, R ug, R kf, R* kabs, R* ksca, R ks) {
  opacity_ks<R>(p, rho, R(p.gam - 1.0) * ug / rho, kf, ks, kabs, ksca);
}
template <typename R>
__device__ __forceinline__ void opacity(const DevParams& p, R rho, R ug, R kf, R* kabs, R* ksca) {
  opacity<R>(p, rho, ug, kf, kabs, ksca, R(p.kscale));
}

// ------------------------------------------------------- face state physics
// U, F^d (12 each) and the gas/radiation signal speeds for one reconstructed
// state at a face: T^d_nu = (w+b^2) u^d u_nu + (p+b^2/2) delta - b^d b_nu,
// R^d_nu = 4/3 Ebar u_r^d u_r_nu + 1/3 Ebar delta; speeds from the fluid-frame
// dispersion (k.u)^2 = c^2 (k.k + (k.u)^2) with k = delta^d - v delta^t
// (Sec. 4.4), gas c^2 = c_s^2 + v_A^2 - c_s^2 v_A^2, radiation
// c^2 = min(1/3, (4/(3 tau))^2) with tau the optical depth of the cell along d.
template <int MET, typename R>
__device__ __forceinline__ void char_speeds(const Geo<MET, R>& g, const R ucon[4], R c2, int d,
                                            R* vmin, R* vmax) {
  R Au = ucon[d], Bu = ucon[0];
  R AA = g.Gdd(d), BB = g.Gtt(), AB = g.Gt(d);
  R qa = Bu * Bu - c2 * (BB + Bu * Bu);
  R qb = R(-2) * (Au * Bu - c2 * (AB + Au * Bu));
  R qc = Au * Au - c2 * (AA + Au * Au);
  R disc = qb * qb - R(4) * qa * qc;
  disc = disc > R(0) ? disc : R(0);
  R sd = sqrt(disc);
  R i2a = R(0.5) / qa;
  R v1 = (-qb + sd) * i2a, v2 = (-qb - sd) * i2a;
  *vmax = v1 > v2 ? v1 : v2;
  *vmin = v1 > v2 ? v2 : v1;
}

template <int MET, typename R>
__device__ __forceinline__ void face_state(const DevParams& p, const Geo<MET, R>& g, int d, R dxd,
                                           R kf, const R P[NPR], R U[NPR], R F[NPR], R sp[4]) {
  const R ks = R(p.kscale);
  R ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq;
  fourvel<MET, R>(g, P[U1], P[U2], P[U3], ucon, ucov, &gm);
  bvec<MET, R>(g, ucon, ucov, P[B1], P[B2], P[B3], bcon, bcov, &bsq);
  const R rho = P[RHO], ug = P[UU];
  const R pg = R(p.gam - 1.0) * ug;
  const R w = rho + ug + pg;
  const R wb = w + bsq, pt = pg + R(0.5) * bsq;
  const R gd = g.gdet;
  const R mt = rho * ucon[0], md = rho * ucon[d];
  U[0] = gd * mt;
  U[1] = gd * (wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + mt);
  U[2] = gd * (wb * ucon[0] * ucov[1] - bcon[0] * bcov[1]);
  U[3] = gd * (wb * ucon[0] * ucov[2] - bcon[0] * bcov[2]);
  U[4] = gd * (wb * ucon[0] * ucov[3] - bcon[0] * bcov[3]);
  U[5] = gd * P[B1];
  U[6] = gd * P[B2];
  U[7] = gd * P[B3];
  F[0] = gd * md;
  F[1] = gd * (wb * ucon[d] * ucov[0] - bcon[d] * bcov[0] + md);
#pragma unroll
  for (int i = 1; i <= 3; ++i)
    F[1 + i] = gd * (wb * ucon[d] * ucov[i] + (i == d ? pt : R(0)) - bcon[d] * bcov[i]);
  const R iut = R(1) / ucon[0];
  const R vd = ucon[d] * iut;
  const R Bd = P[B1 + d - 1];
#pragma unroll
  for (int i = 1; i <= 3; ++i) F[4 + i] = (i == d) ? R(0) : gd * (P[B1 + i - 1] * vd - Bd * ucon[i] * iut);
  // radiation
  R urc[4], urv[4], gr;
  fourvel<MET, R>(g, P[UR1], P[UR2], P[UR3], urc, urv, &gr);
  const R E = P[ER];
  const R e43 = R(4.0 / 3.0) * E, e13 = E * R(1.0 / 3.0);
  U[8] = gd * (e43 * urc[0] * urv[0] + e13);
  U[9] = gd * (e43 * urc[0] * urv[1]);
  U[10] = gd * (e43 * urc[0] * urv[2]);
  U[11] = gd * (e43 * urc[0] * urv[3]);
#pragma unroll
  for (int n = 0; n < 4; ++n) F[8 + n] = gd * (e43 * urc[d] * urv[n] + (n == d ? e13 : R(0)));
  // gas fast magnetosonic speed
  R cs2 = R(p.gam) * pg / w;
  R va2 = bsq / (w + bsq);
  R cms2 = cs2 + va2 - cs2 * va2;
  cms2 = cms2 > R(1) ? R(1) : (cms2 < R(0) ? R(0) : cms2);
  char_speeds<MET, R>(g, ucon, cms2, d, &sp[0], &sp[1]);
  R kabs, ksca;
  opacity<R>(p, rho, ug, kf, &kabs, &ksca, ks);
  R tau = (kabs + ksca) * sqrt(g.gdd(d)) * dxd;
  R cr2 = R(1.0 / 3.0);
  if (tau > R(0)) {
    R lim = R(4.0 / 3.0) / tau;
    lim = lim * lim;
    cr2 = lim < cr2 ? lim : cr2;
  }
  char_speeds<MET, R>(g, urc, cr2, d, &sp[2], &sp[3]);
}

// Gas and radiation signal speeds (vmin, vmax) of one reconstructed state;
// dl = sqrt(g_dd) dx^d is the proper length of the cell along d (the same for
// both states of a face) and kf the per-zone opacity of the state's cell.
// lor (optional) returns the gas and radiation Lorentz factors and 1/u^t for
// face_accum.  b^2 = (B^i B_i + (B^i u_i)^2) / (u^t)^2 (the identity behind
// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t), without forming b^mu.
template <int MET, typename R>
__device__ __forceinline__ void face_speeds(const DevParams& p, const Geo<MET, R>& g, int d, R dl,
                                            R kf, R ks, const R P[NPR], R sp[4], unsigned* code = nullptr,
                                            R* lor = nullptr) {
  R ucon[4], ucov[4], gm;
  fourvel<MET, R>(g, P[U1], P[U2], P[U3], ucon, ucov, &gm);
  const R Bu = P[B1] * ucov[1] + P[B2] * ucov[2] + P[B3] * ucov[3];
  const R iut = g.alpha / gm;
  const R bsq = (g.sq3(P[B1], P[B2], P[B3]) + Bu * Bu) * iut * iut;
  const R rho = P[RHO], ug = P[UU];
  const R pg = R(p.gam - 1.0) * ug;
  const R w = rho + ug + pg;
  R cs2, va2;
  if constexpr (std::is_same<R, double>::value) {  // one division (w^2 stays in FP64's range)
    const R iw = R(1) / (w * (w + bsq));
    cs2 = R(p.gam) * pg * (w + bsq) * iw;
    va2 = bsq * w * iw;
  } else {
    cs2 = R(p.gam) * pg / w;
    va2 = bsq / (w + bsq);
  }
  R cms2 = cs2 + va2 - cs2 * va2;
  if (code) *code = (cms2 > R(1) ? 1u : 0u) | (cms2 < R(0) ? 2u : 0u);
  cms2 = cms2 > R(1) ? R(1) : (cms2 < R(0) ? R(0) : cms2);
  char_speeds<MET, R>(g, ucon, cms2, d, &sp[0], &sp[1]);
  R urc[4], urv[4], gr;
  fourvel<MET, R>(g, P[UR1], P[UR2], P[UR3], urc, urv, &gr);
  if (lor) {
    lor[0] = gm;
    lor[1] = gr;
    lor[2] = iut;
  }
  R kabs, ksca;
  opacity<R>(p, rho, ug, kf, &kabs, &ksca, ks);
  R tau = (kabs + ksca) * dl;
  R cr2 = R(1.0 / 3.0);
  if (tau > R(0)) {
    R lim = R(4.0 / 3.0) / tau;
    lim = lim * lim;
    if (code && lim < cr2) *code |= 4u;
    cr2 = lim < cr2 ? lim : cr2;
  }
  char_speeds<MET, R>(g, urc, cr2, d, &sp[2], &sp[3]);
}

// out[q] += aF_q F_q + aU_q U_q for one reconstructed state, with (aF, aU)
// taking the gas values for q < 8 and the radiation values for q >= 8.  HLL
// and LAXF are linear in (F_L, U_L, F_R, U_R), so each state adds its own
// share and the two states' U and F never need to be held together.  lor
// (optional): the state's gas and radiation Lorentz factors and 1/u^t from
// face_speeds.
template <int MET, typename R>
__device__ __forceinline__ void face_accum(const DevParams& p, const Geo<MET, R>& g, int d,
                                           const R P[NPR], R aFg, R aUg, R aFr, R aUr, R out[NPR],
                                           R* fs = nullptr, const R* lor = nullptr) {
  R ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq;
  if (lor) {
    gm = lor[0];
    fourvel_g<MET, R>(g, P[U1], P[U2], P[U3], gm, ucon, ucov);
  } else {
    fourvel<MET, R>(g, P[U1], P[U2], P[U3], ucon, ucov, &gm);
  }
  const R iut = lor ? lor[2] : g.alpha / gm;
  bvec_iut<MET, R>(g, ucon, ucov, iut, P[B1], P[B2], P[B3], bcon, bcov, &bsq);
  const R rho = P[RHO], ug = P[UU];
  const R pg = R(p.gam - 1.0) * ug;
  const R wb = rho + ug + pg + bsq, pt = pg + R(0.5) * bsq;
  const R gd = g.gdet;
  const R mt = rho * ucon[0], md = rho * ucon[d];
  out[0] += gd * (aFg * md + aUg * mt);
  // entropy flux sqrt(-g) S u^d = s_gas times the mass flux (Sec. 2, Eq. S)
  if (fs) *fs += entropy_per_baryon<R>(p, rho, ug) * (gd * (aFg * md + aUg * mt));
  out[1] += gd * (aFg * (wb * ucon[d] * ucov[0] - bcon[d] * bcov[0] + md) +
                  aUg * (wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + mt));
#pragma unroll
  for (int i = 1; i <= 3; ++i)
    out[1 + i] += gd * (aFg * (wb * ucon[d] * ucov[i] + (i == d ? pt : R(0)) - bcon[d] * bcov[i]) +
                        aUg * (wb * ucon[0] * ucov[i] - bcon[0] * bcov[i]));
  const R vd = ucon[d] * iut;
  const R Bd = P[B1 + d - 1];
#pragma unroll
  for (int i = 1; i <= 3; ++i) {
    R f = (i == d) ? R(0) : (P[B1 + i - 1] * vd - Bd * ucon[i] * iut);
    out[4 + i] += gd * (aFg * f + aUg * P[B1 + i - 1]);
  }
  R urc[4], urv[4], gr;
  if (lor) fourvel_g<MET, R>(g, P[UR1], P[UR2], P[UR3], lor[1], urc, urv);
  else fourvel<MET, R>(g, P[UR1], P[UR2], P[UR3], urc, urv, &gr);
  const R E = P[ER];
  const R e43 = R(4.0 / 3.0) * E, e13 = E * R(1.0 / 3.0);
#pragma unroll
  for (int n = 0; n < 4; ++n)
    out[8 + n] += gd * (aFr * (e43 * urc[d] * urv[n] + (n == d ? e13 : R(0))) +
                        aUr * (e43 * urc[0] * urv[n] + (n == 0 ? e13 : R(0))));
}

// ------------------------------------------------------ M1 inversion (FP64)
// Closed form in the ZAMO frame (Sec. 4.6): E_rad = alpha^2 R^{tt},
// U~^i = alpha g^{i mu} R^t_mu + E_rad alpha g^{ti}, y = U~^2/E_rad^2,
// gamma^2 = (2 - y + sqrt(4-3y)) / (4(1-y)), p_rad = E_rad/(4 gamma^2 - 1),
// u~^i = gamma U~^i / (4 p_rad gamma^2).  Limiters: BASIC (lim 0) and TYPE2
// (lim 2).  Returns 1 if E_rad <= 0 on entry.
template <int MET, typename T = double>
__device__ __forceinline__ int rad_invert(const DevParams& p, const Geo<MET, T>& g, const T Rt[4], int lim,
                                          T out[4], int* limited = nullptr) {
  const T a = g.alpha;
  T Erad = a * a * g.raise_t(Rt);
  T Ut[3];
  g.raise3(Rt, Ut);
  const T et = Erad * g.Gt(1);
  Ut[0] = a * (Ut[0] + et);
  Ut[1] = a * Ut[1];
  Ut[2] = a * Ut[2];
  T Utsq = g.sq3(Ut[0], Ut[1], Ut[2]);
  const double ymax = p.ymax_rad;
  int negE = Erad <= 0.0;
  T y;
  if (lim == 0) {
    if (Erad <= 0.0) {
      out[0] = T(1e-300);
      out[1] = out[2] = out[3] = T(0.0);
      return negE;
    }
    y = Utsq > 0.0 ? Utsq / (Erad * Erad) : T(0.0);  // no momentum: y = 0 (Erad^2 may underflow)
    if (y < 0.0) {
      y = T(0.0);
      Ut[0] = Ut[1] = Ut[2] = T(0.0);
    }
    if (y > ymax) {
      T f = sqrt(T(ymax) / y);
      Ut[0] *= f;
      Ut[1] *= f;
      Ut[2] *= f;
      y = T(ymax);
    }
  } else {
    y = Erad > 0.0 ? (Utsq > 0.0 ? Utsq / (Erad * Erad) : T(0.0)) : T(HUGE_VAL);
    if (limited) *limited = (Erad <= 0.0 || y > ymax) ? 1 : 0;
    if (Erad <= 0.0 || y > ymax) {
      Erad = T(1e-150) + sqrt(Utsq / T(ymax));
      y = Utsq / (Erad * Erad);
    }
    if (y < 0.0) y = T(0.0);
  }
  // With s = sqrt(4 - 3y), Eq. gammarvsy gives gamma^2 = (s+2)/(4(s-1)) and
  // 4 gamma^2 - 1 = 3/(s-1), so Ebar = 3 p_rad = E_rad (s-1) and
  // u~^i = gamma U~^i/(4 p_rad gamma^2) = 3 U~^i / (2 E_rad sqrt((s+2)(s-1))).
  const T sq = sqrt(T(4.0) - T(3.0) * y);
  const T sm1 = sq - T(1.0);
  out[0] = Erad * sm1;
  T f = T(1.5) / Erad * rsqrt_<T>((sq + T(2.0)) * sm1);
  out[1] = f * Ut[0];
  out[2] = f * Ut[1];
  out[3] = f * Ut[2];
  return negE;
}

// ---------------------------------------------------- gas 1D_W inversion (FP64)
// Sec. 4.5: Newton on f(W') = W' - E' - p + B^2 (1+v~^2)/2 - S^2/(2W^2) with
// W = W' + D, v~^2 from Eq. vsqeq, then v~^i from Eq. tveq.  Input in
// conserved form: Dlab = rho0 u^t, taue = T^t_t + rho0 u^t, Tt[3] = T^t_i,
// B[3] lab field; guess primitives give the starting W'.  Writes rho0, u_g,
// u~^i into out[0..4].  Returns 0 on success.
template <int MET>
__device__ __forceinline__ int gas_invert(const DevParams& p, const Geo<MET, double>& g, double Dlab,
                                          double taue, const double Tt[3], const double B[3],
                                          const double* Pg, double tol, double out[5]) {
  const double a = g.alpha, gam = p.gam;
  const double D = a * Dlab;
  const double Ttt = taue - Dlab;
  double Ep = -taue + (1.0 - a) * Dlab + a * a * g.Gt(1) * Tt[0];
  const double E = Ep + D;
  double Q[4] = {a * Ttt, a * Tt[0], a * Tt[1], a * Tt[2]};
  double Qt[3];
  g.raise3(Q, Qt);
  Qt[0] += E * a * g.Gt(1);
  const double Bz0 = a * B[0], Bz1 = a * B[1], Bz2 = a * B[2];
  const double QdB = Q[1] * Bz0 + Q[2] * Bz1 + Q[3] * Bz2;
  const double Bsq = g.sq3(Bz0, Bz1, Bz2);
  const double Qtsq = g.sq3(Qt[0], Qt[1], Qt[2]);
  const double S2 = QdB * QdB;
  if (!(D > 0.0) || !isfinite(E)) return 1;
  double q0 = g.sq3(Pg[U1], Pg[U2], Pg[U3]);
  double gm0 = sqrt(1.0 + q0);
  double ugg = Pg[UU] > 0.0 ? Pg[UU] : 0.0;
  double Wp = D * q0 / (1.0 + gm0) + gam * ugg * gm0 * gm0;
  if (!(Wp > 0.0)) Wp = fmax(fabs(Ep), 1e-300);
  const double gfac = (gam - 1.0) / gam;
  double f = 0.0, df = 0.0;
  auto resid = [&](double Wpv, double* fo, double* dfo) -> bool {
    double W = Wpv + D;
    double WB = Bsq + W;
    double iW = 1.0 / W, iWB = 1.0 / WB;
    double vsq = (Qtsq * W * W + S2 * (Bsq + 2.0 * W)) * (iWB * iWB) * (iW * iW);
    if (!(vsq < 1.0) || !(W > 0.0)) return false;
    double g2 = 1.0 / (1.0 - vsq);
    double gg = sqrt(g2);
    double usq = g2 * vsq;
    double chi = (Wpv - D * usq / (gg + 1.0)) * (1.0 - vsq);
    double pg = gfac * chi;
    *fo = Wpv - Ep - pg + 0.5 * Bsq * (1.0 + vsq) - 0.5 * S2 * iW * iW;
    double iW3 = iW * iW * iW, iWB3 = iWB * iWB * iWB;
    double dvsq = -2.0 * iW3 * iWB3 * (S2 * (3.0 * W * WB + Bsq * Bsq) + Qtsq * W * W * W);
    double dchi = (1.0 - vsq) - W * dvsq + 0.5 * D * gg * dvsq;
    *dfo = 1.0 - gfac * dchi + 0.5 * Bsq * dvsq + S2 * iW3;
    return true;
  };
  int guard = 0;
  while (!resid(Wp, &f, &df) && guard < 200) {
    Wp = 2.0 * Wp + 1e-300;
    ++guard;
  }
  if (guard >= 200) return 2;
  bool conv = false;
  for (int it = 0; it < 50; ++it) {
    if (!(df != 0.0) || !isfinite(f) || !isfinite(df)) return 3;
    double dW = -f / df;
    double Wn = Wp + dW, fn = 0.0, dfn = 0.0;
    int back = 0;
    while ((!(Wn > 0.0) || !resid(Wn, &fn, &dfn)) && back < 60) {
      dW *= 0.5;
      Wn = Wp + dW;
      ++back;
    }
    if (back >= 60) return 4;
    Wp = Wn;
    f = fn;
    df = dfn;
    if (fabs(dW) <= tol * fabs(Wp)) {
      conv = true;
      break;
    }
  }
  if (!conv) return 5;
  double W = Wp + D;
  double vsq = (Qtsq * W * W + S2 * (Bsq + 2.0 * W)) / ((Bsq + W) * (Bsq + W) * W * W);
  double g2 = 1.0 / (1.0 - vsq);
  double gg = sqrt(g2);
  double usq = g2 * vsq;
  double chi = (Wp - D * usq / (gg + 1.0)) / g2;
  double rho = D / gg, ug = chi / gam;
  if (!(rho > 0.0) || !(ug > 0.0) || !isfinite(ug)) return 6;
  out[0] = rho;
  out[1] = ug;
  double iv = gg / (W + Bsq), sb = QdB / W;
  out[2] = iv * (Qt[0] + sb * Bz0);
  out[3] = iv * (Qt[1] + sb * Bz1);
  out[4] = iv * (Qt[2] + sb * Bz2);
  return 0;
}

}  // namespace hr
