// Jacobian of the PMHD error function on the FP32 pipe (forward-mode tangents).
//
// The PMHD Newton iteration (Sec. 4.9, Eq. newton) needs J = dE_gas/dx at the
// iterate x = (u_g, u~^1, u~^2, u~^3).  The error E itself, and with it the
// stopping test and the root that is accepted, stays in FP64 (hr_implicit.cuh);
// the Jacobian only sets how fast the iteration converges.  On this chip an
// FP64 instruction issues at 1/64 of the FP32 rate, so the four extra FP64
// residual evaluations of a finite-difference Jacobian were half of the update
// kernel's FP64 work.  Here each column of J is the exact derivative of the
// same error function along one unknown, evaluated in FP32 with a value and
// one derivative per quantity (the register footprint of one FP64 pass); the
// radiation R^t_nu, which the error recovers from total conservation as a
// difference of large numbers, takes its value from the FP64 evaluation at the
// same iterate and only its derivative from FP32.  The columns carry FP32
// round-off (about 1e-6 relative) where finite differences with offset 1e-8
// carry about 1e-8: either way Newton converges to the FP64 root.
//
// The operations follow pmhd_res line by line: fourvel, bvec_iut, T^t_nu, the
// TYPE2 M1 inversion of Sec. 4.6, the radiation 4-velocity, the opacity and the
// four-force of Eq. Gcov in its rank-one-plus-isotropic form.
#pragma once
#include "hr_phys.cuh"

namespace hr {

// FP32 value with one directional derivative.  Every operation is an
// explicitly rounded intrinsic, which the compiler may not contract into a
// different multiply-add: the Jacobian is then the same bits in every kernel
// that evaluates it (the update kernel and the Newton continuation kernel).
struct F1 {
  float v, d;
};
__device__ __forceinline__ F1 fc(float v) { return F1{v, 0.0f}; }
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1{__fadd_rn(a.v, b.v), __fadd_rn(a.d, b.d)}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1{__fsub_rn(a.v, b.v), __fsub_rn(a.d, b.d)}; }
__device__ __forceinline__ F1 operator-(F1 a) { return F1{-a.v, -a.d}; }
__device__ __forceinline__ F1 operator+(F1 a, float b) { return F1{__fadd_rn(a.v, b), a.d}; }
__device__ __forceinline__ F1 operator+(float a, F1 b) { return F1{__fadd_rn(a, b.v), b.d}; }
__device__ __forceinline__ F1 operator-(F1 a, float b) { return F1{__fsub_rn(a.v, b), a.d}; }
__device__ __forceinline__ F1 operator-(float a, F1 b) { return F1{__fsub_rn(a, b.v), -b.d}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) {
  return F1{__fmul_rn(a.v, b.v), __fmaf_rn(a.d, b.v, __fmul_rn(a.v, b.d))};
}
__device__ __forceinline__ F1 operator*(F1 a, float b) { return F1{__fmul_rn(a.v, b), __fmul_rn(a.d, b)}; }
__device__ __forceinline__ F1 operator*(float a, F1 b) { return F1{__fmul_rn(a, b.v), __fmul_rn(a, b.d)}; }
__device__ __forceinline__ F1 operator/(F1 a, F1 b) {
  const float ib = __fdiv_rn(1.0f, b.v), q = __fmul_rn(a.v, ib);
  return F1{q, __fmul_rn(__fsub_rn(a.d, __fmul_rn(q, b.d)), ib)};
}
__device__ __forceinline__ F1 operator/(float a, F1 b) {
  const float ib = __fdiv_rn(1.0f, b.v), q = __fmul_rn(a, ib);
  return F1{q, __fmul_rn(__fmul_rn(-q, b.d), ib)};
}
__device__ __forceinline__ F1 fsqrt(F1 a) {
  const float s = __fsqrt_rn(a.v);
  return F1{s, s > 0.0f ? __fdiv_rn(__fmul_rn(0.5f, a.d), s) : 0.0f};
}
__device__ __forceinline__ F1 frsqrt(F1 a) {
  const float s = rsqrtf(a.v);
  return F1{s, __fmul_rn(__fmul_rn(__fmul_rn(-0.5f, s), __fmul_rn(s, s)), a.d)};
}

// FP32 copy of the metric components the error function uses.
template <int MET>
struct GeoF {
  float g00, g01, g03, g11, g13, g22, g33;
  float G00, G01, G11, G13, G22, G33;
  float alpha, ialpha;
  __device__ __forceinline__ GeoF() {}  // Minkowski: the forms below read no component
  // from the 15 staged components (TanStage: g00 .. ialpha in this order)
  __device__ __forceinline__ explicit GeoF(const volatile float* a)
      : g00(a[0]), g01(a[1]), g03(a[2]), g11(a[3]), g13(a[4]), g22(a[5]), g33(a[6]), G00(a[7]), G01(a[8]),
        G11(a[9]), G13(a[10]), G22(a[11]), G33(a[12]), alpha(a[13]), ialpha(a[14]) {}
  __device__ __forceinline__ void lower(const F1 v[4], F1 w[4]) const {
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
  __device__ __forceinline__ F1 sq3(F1 a, F1 b, F1 c) const {
    if constexpr (MET == MINK) return a * a + b * b + c * c;
    else return g11 * (a * a) + g22 * (b * b) + g33 * (c * c) + (2.0f * g13) * (a * c);
  }
};

// 4-velocity from the ZAMO-relative spatial components (fourvel).
template <int MET>
__device__ __forceinline__ void fourvel_t(const GeoF<MET>& g, F1 q1, F1 q2, F1 q3, F1 ucon[4], F1 ucov[4], F1* gm) {
  *gm = fsqrt(1.0f + g.sq3(q1, q2, q3));
  if constexpr (MET == MINK) {
    ucon[0] = *gm;
    ucon[1] = q1;
  } else {
    ucon[0] = *gm * g.ialpha;
    ucon[1] = q1 - *gm * (g.alpha * g.G01);
  }
  ucon[2] = q2;
  ucon[3] = q3;
  g.lower(ucon, ucov);
}

// FP32 inputs of the Kerr-Schild tangent passes, staged in thread-local memory: the 15
// metric components of GeoF (v[0..14]), the zone's rho0 u^t, 1/(rho0 u^t), B,
// step h and opacity inputs (v[15..23]), converted once per solve, and the
// iterate's unknowns x and R^t_nu of the FP64 error function (v[24..31]),
// converted once per Jacobian.  Every column pass loads them from here: a
// conversion runs on the FP64 pipe, and the compiler, short of registers,
// would otherwise convert them again in each of the four passes.  The zone
// part is filled at the solve's first Jacobian (zone = 1 from then on), so a
// solve that converges without one converts nothing.
struct TanStage {
  volatile float v[32];
  int zone = 0;
};

template <int MET, class Sys>
__device__ __forceinline__ void tan_stage_zone(const Sys& s, TanStage& ts) {
  const auto& g = s.g;
  const double m[15] = {g.g00, g.g01, g.g03, g.g11, g.g13, g.g22, g.g33, g.G00,
                        g.G01, g.G11, g.G13, g.G22, g.G33, g.alpha, g.ialpha};
#pragma unroll
  for (int i = 0; i < 15; ++i) ts.v[i] = (float)m[i];
  const double c[8] = {s.Dlab, s.iDlab, s.B[0], s.B[1], s.B[2], s.h, s.ks, s.kf};
#pragma unroll
  for (int i = 0; i < 8; ++i) ts.v[15 + i] = (float)c[i];
  ts.zone = 1;
}

// the FP32 inputs of one column pass: from the staged copy (v[15..31]), or,
// on the Minkowski path, which has no metric to stage, converted in registers
struct TanIn {
  float x[4], rt[4], Dlab, iDlab, B[3], h, ks, kf;
  template <class Sys>
  __device__ __forceinline__ TanIn(const Sys& s, const double xd[4], const double Rt64[4])
      : Dlab((float)s.Dlab), iDlab((float)s.iDlab), B{(float)s.B[0], (float)s.B[1], (float)s.B[2]},
        h((float)s.h), ks((float)s.ks), kf((float)s.kf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] = (float)xd[i];
      rt[i] = (float)Rt64[i];
    }
  }
  __device__ __forceinline__ explicit TanIn(const TanStage& ts)
      : Dlab(ts.v[15]), iDlab(ts.v[16]), B{ts.v[17], ts.v[18], ts.v[19]}, h(ts.v[20]), ks(ts.v[21]),
        kf(ts.v[22]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] = ts.v[24 + i];
      rt[i] = ts.v[28 + i];
    }
  }
};

// Column j of the PMHD Jacobian dE_gas/dx at x (inputs in ti).  Returns false
// if a value is not finite.
template <int MET>
__device__ __forceinline__ bool pmhd_jac_column(const DevParams& p, const TanIn& ti, const GeoF<MET>& g, int j,
                                                float col[4]) {
  F1 X[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) X[i] = F1{ti.x[i], i == j ? 1.0f : 0.0f};
  const float gm1 = p.gm1f;
  F1 ucon[4], ucov[4], gm;
  fourvel_t<MET>(g, X[1], X[2], X[3], ucon, ucov, &gm);
  const F1 iut = (MET == MINK ? 1.0f : g.alpha) / gm;
  const F1 rho = ti.Dlab * iut;
  const float B1 = ti.B[0], B2 = ti.B[1], B3 = ti.B[2];
  F1 bcon[4], bcov[4];
  const F1 bt = B1 * ucov[1] + B2 * ucov[2] + B3 * ucov[3];
  bcon[0] = bt;
  bcon[1] = (B1 + bt * ucon[1]) * iut;
  bcon[2] = (B2 + bt * ucon[2]) * iut;
  bcon[3] = (B3 + bt * ucon[3]) * iut;
  g.lower(bcon, bcov);
  const F1 bsq = bcon[0] * bcov[0] + bcon[1] * bcov[1] + bcon[2] * bcov[2] + bcon[3] * bcov[3];
  const F1 pg = gm1 * X[0];
  const F1 wb = rho + X[0] + pg + bsq, pt = pg + 0.5f * bsq;
  F1 Tc[4];
  Tc[0] = wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + rho * ucon[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) Tc[k] = wb * ucon[0] * ucov[k] - bcon[0] * bcov[k];
  // R^t_nu = R*^t_nu - (T^t_nu(x) - T*^t_nu): FP64 value, derivative -dT
  F1 Rt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Rt[k] = F1{ti.rt[k], -Tc[k].d};
  // TYPE2 M1 inversion (Sec. 4.6)
  F1 Erad, Ut[3];
  if constexpr (MET == MINK) {
    Erad = -Rt[0];
    Ut[0] = Rt[1];
    Ut[1] = Rt[2];
    Ut[2] = Rt[3];
  } else {
    const float a = g.alpha;
    Erad = (a * a) * (g.G00 * Rt[0] + g.G01 * Rt[1]);
    Ut[0] = a * (g.G01 * Rt[0] + g.G11 * Rt[1] + g.G13 * Rt[3] + Erad * g.G01);
    Ut[1] = a * (g.G22 * Rt[2]);
    Ut[2] = a * (g.G13 * Rt[1] + g.G33 * Rt[3]);
  }
  const F1 Utsq = g.sq3(Ut[0], Ut[1], Ut[2]);
  const float ymax = p.ymaxf;
  F1 y;
  if (Erad.v > 0.0f) {
    // y = U~^2 / E_rad^2 from the ratios (E_rad^2 can underflow in FP32)
    const F1 ie = 1.0f / Erad;
    y = Utsq.v > 0.0f ? g.sq3(Ut[0] * ie, Ut[1] * ie, Ut[2] * ie) : fc(0.0f);
  } else {
    y = fc(HUGE_VALF);
  }
  if (Erad.v <= 0.0f || y.v > ymax) {
    // the limiter sets E_rad so that y = y_max: y is then constant
    Erad = fsqrt(Utsq * (1.0f / ymax));
    y = fc(ymax);
  }
  if (y.v < 0.0f) y = fc(0.0f);
  const F1 sq = fsqrt(4.0f - 3.0f * y);
  const F1 sm1 = sq - 1.0f;
  const F1 E = Erad * sm1;
  const F1 f = (1.5f / Erad) * frsqrt((sq + 2.0f) * sm1);
  F1 urc[4], urv[4], gr;
  fourvel_t<MET>(g, f * Ut[0], f * Ut[1], f * Ut[2], urc, urv, &gr);
  // gas temperature T = (gamma-1) u_g u^t / (rho0 u^t)
  const F1 Tg = (gm1 * ti.iDlab) * (X[0] * ucon[0]);
  // opacities (opacity_ks)
  const float ks = ti.ks;
  F1 kabs;
  if (p.opacity == 2) {
    kabs = fc(ks * ti.kf);
  } else if (p.opacity == 1) {
    const float Tmin = p.Tminf;
    const F1 Tcl = Tg.v > Tmin ? Tg : fc(Tmin);
    const F1 t35 = frsqrt(Tcl) / (Tcl * Tcl * Tcl);  // T^-3.5 without forming T^7
    kabs = (ks * p.kabs0f) * (rho * rho) * t35;
  } else {
    kabs = (ks * p.kabs0f) * rho;
  }
  const F1 ksca = (ks * p.kes0f) * rho;
  // four-force (four_force_rad)
  const F1 T2 = Tg * Tg;
  const F1 lam = kabs * p.aradf * (T2 * T2);
  const F1 uru = urv[0] * ucon[0] + urv[1] * ucon[1] + urv[2] * ucon[2] + urv[3] * ucon[3];
  const F1 c1 = (4.0f / 3.0f) * E * uru, c2 = E * (1.0f / 3.0f);
  const F1 uRu = c1 * uru - c2;
  const F1 kt = kabs + ksca;
  const F1 A = -(kt * c1);
  const F1 C = -(kt * c2 + lam + ksca * uRu);
  const float h = ti.h;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const F1 G = A * urv[k] + C * ucov[k];
    col[k] = __fsub_rn(Tc[k].d, __fmul_rn(h, G.d));
    ok = ok && isfinite(col[k]);
  }
  return ok;
}

// The PMHD Jacobian (J[i][c] = dE_i/dx_c) from four FP32 tangent passes; ts
// holds the solve's staged inputs (tan_stage_zone; Kerr-Schild only).
__device__ __forceinline__ void jac_store_column(double J[4][4], int j, const float col[4]) {
  // column j written through compile-time indices
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (c == j) J[i][c] = (double)col[i];
}

template <int MET, class Sys>
__device__ __forceinline__ bool pmhd_jacobian_fp32(const DevParams& p, const Sys& s, TanStage& ts,
                                                   const double x[4], const double Rt64[4], double J[4][4]) {
  bool ok = true;
  if constexpr (MET == MINK) {
    const TanIn ti(s, x, Rt64);
    const GeoF<MET> g;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      float col[4];
      ok = pmhd_jac_column<MET>(p, ti, g, j, col) && ok;
      jac_store_column(J, j, col);
    }
  } else {
    if (!ts.zone) tan_stage_zone<MET>(s, ts);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ts.v[24 + i] = (float)x[i];
      ts.v[28 + i] = (float)Rt64[i];
    }
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      float col[4];
      ok = pmhd_jac_column<MET>(p, TanIn(ts), GeoF<MET>(ts.v), j, col) && ok;
      jac_store_column(J, j, col);
    }
  }
  return ok;
}

}  // namespace hr
