// Implicit gas-radiation four-force solve of one zone (FP64), Sec. 4.7-4.10
// of McKinney et al. (2014).
//
// Solves T^t_nu(x) - T*^t_nu = h G_nu(x) (Eq. source3) with rho0 u^t and B
// fixed and the radiation taken from total energy-momentum conservation.
// PMHD iterates the gas primitives x = (u_g, u~^i); URAD iterates x = R^t_nu
// and PRAD x = (Ebar, u~^i_rad), both recovering the gas from a 1D_W
// inversion inside every residual.  Newton
// steps follow Eq. newton with D = 1.  The PMHD Jacobian is the exact
// derivative of the error function evaluated on the FP32 pipe
// (hr_tangent.cuh); it falls back to the paper's finite differences (FP64,
// one-sided; the paper's two-sided PMHD differences belong to its staged
// scheme, which is not used; normalised offset 1e-8, switching to 1e-10 once
// e_I < 1e-9) for the rest of a solve when the FP32 Jacobian is not finite or
// singular, or when a step taken with it raised e_T.  URAD and PRAD
// use the finite differences.  The error, and with it every stopping rule of
// Sec. 4.10 (tolerance, stalled error, repeated rises, tiny step, step limit)
// and the best-error bookkeeping, is FP64.
//
// The four-force uses the rank-one-plus-isotropic form of the M1 tensor:
// R^mu_a u^a = 4/3 Ebar (u_r.u) u_r^mu + 1/3 Ebar u^mu, so G_nu (Eq. Gcov) is a
// combination of u_r_nu and u_nu and needs no 4x4 contraction.
#pragma once
#include "hr_phys.cuh"
#include "hr_tangent.cuh"

namespace hr {

// The implicit system of one zone.  T is double in the step; the adjoint
// evaluates the same functions on dual numbers.
template <int MET, typename T = double>
struct ImpSysT {
  Geo<MET, T> g;
  T Dlab;   // rho0 u^t
  T iDlab;  // 1 / (rho0 u^t)
  T Ts[4];  // explicit T^t_nu, rest-mass flux added to the t row
  T Rs[4];  // explicit R^t_nu
  T B[3];
  T h;      // b_s dt
  T kf;     // the zone's absorption opacity when it is a per-zone field
  T ks;     // global opacity scale kappa_scale
  T sgk[3]; // sqrt(gamma^{kk}) of the ZAMO slice
  bool entropy;  // the entropy equation replaces the gas energy row (Eq. source6)
  T Sstar;       // explicit S u^t (the conserved entropy over sqrt(-g))
  bool cold;     // cold MHD (Sec. 4.11): u_g held, the momentum rows only
};
template <int MET>
using ImpSys = ImpSysT<MET, double>;

template <typename T = double>
struct ImpResT {
  T Eg[4], Er[4];
  T eT, eI;
  T eg0;  // normalised error of the gas energy (or entropy) row alone
  T er0;  // normalised error of the radiation energy row alone
  int negE;
  bool ok;
};
using ImpRes = ImpResT<double>;

// Gas and radiation state of an iterate: the pieces of the residual that the
// final primitives need.
template <typename T = double>
struct ImpStateT {
  T rho, ug, Pr[4];
  T Rt_pre[4];
  int negE;  // the TYPE2 inversion saw E_rad <= 0
};
using ImpState = ImpStateT<double>;

// G_nu for gas temperature T (given, so the caller can form it without a
// division).
template <int MET, typename T = double>
__device__ __forceinline__ void four_force_rad(const DevParams& p, T rho, T Tg, T kf, T ks, const T ucon[4],
                                               const T ucov[4], const T urc[4], const T urv[4], T E,
                                               T G[4]) {
  T kabs, ksca;
  opacity_ks<T>(p, rho, Tg, kf, ks, &kabs, &ksca);
  T T2 = Tg * Tg;
  T lam = kabs * p.a_rad * T2 * T2;
  T uru = urv[0] * ucon[0] + urv[1] * ucon[1] + urv[2] * ucon[2] + urv[3] * ucon[3];
  T c1 = (4.0 / 3.0) * E * uru, c2 = E * (1.0 / 3.0);
  T uRu = c1 * uru - c2;
  T kt = kabs + ksca;
  T A = -kt * c1;
  T C = -(kt * c2 + lam + ksca * uRu);
  (void)urc;
#pragma unroll
  for (int n = 0; n < 4; ++n) G[n] = A * urv[n] + C * ucov[n];
}

template <int MET, typename T = double>
__device__ __forceinline__ void normalise(const ImpSysT<MET, T>& s, const T Tc[4], const T Rc[4],
                                          const T G[4], bool iter_gas, ImpResT<T>& r, T eS = T(-1.0),
                                          T eSr = T(-1.0)) {
  T dg0 = fabs(Tc[0]) + fabs(s.Ts[0]) + s.h * fabs(G[0]);
  T dr0 = fabs(Rc[0]) + fabs(s.Rs[0]) + s.h * fabs(G[0]);
  T dgs = T(0.0), drs = T(0.0);
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    dgs += s.sgk[k - 1] * (fabs(Tc[k]) + fabs(s.Ts[k]) + s.h * fabs(G[k]));
    drs += s.sgk[k - 1] * (fabs(Rc[k]) + fabs(s.Rs[k]) + s.h * fabs(G[k]));
  }
  // the spatial norm also carries the energy-row terms (momentum is bounded
  // by energy; a field at rest must not divide round-off by round-off)
  dgs += dg0;
  drs += dr0;
  T eg[4], er[4];
  eg[0] = dg0 > 0.0 ? fabs(r.Eg[0]) / dg0 : T(0.0);
  er[0] = dr0 > 0.0 ? fabs(r.Er[0]) / dr0 : T(0.0);
  T idgs = dgs > 0.0 ? 1.0 / dgs : T(0.0), idrs = drs > 0.0 ? 1.0 / drs : T(0.0);
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    eg[k] = fabs(r.Eg[k]) * s.sgk[k - 1] * idgs;
    er[k] = fabs(r.Er[k]) * s.sgk[k - 1] * idrs;
  }
  if (r.negE) eg[0] = er[0] = T(0.0);
  if (eS >= 0.0) {  // entropy row in place of the gas energy row; the radiation energy row drops
    eg[0] = r.negE ? T(0.0) : eS;  // excluded after a TYPE2 negative energy (Sec. 4.10)
    er[0] = T(0.0);
  }
  if (eSr >= 0.0) {  // the radiation methods' entropy row (the energy rows drop)
    eg[0] = T(0.0);
    er[0] = r.negE ? T(0.0) : eSr;
  }
  r.eg0 = eg[0];
  r.er0 = er[0];
  if (s.cold) {  // cold MHD: energy and entropy ignored, the mean of the momentum rows
    T cT = T(0.0), cI = T(0.0);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      cT += fmax(eg[k], er[k]);
      cI += eg[k];
    }
    r.eT = cT / 3.0;
    r.eI = cI / 3.0;
    return;
  }
  T sT = T(0.0), sI = T(0.0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    sT += fmax(eg[k], er[k]);
    sI += iter_gas ? eg[k] : er[k];
  }
  r.eT = 0.25 * sT;
  r.eI = 0.25 * sI;
}

// PMHD error function.  With norm == false only Eg is formed (Jacobian columns).
template <class X>
struct nondeduced {
  using type = X;
};

template <int MET, typename T = double>
__device__ __forceinline__ void pmhd_res(const DevParams& p, const ImpSysT<MET, T>& s, const T x[4],
                                         ImpResT<T>& r, typename nondeduced<ImpStateT<T>>::type* st,
                                         bool norm) {
  const auto& g = s.g;
  T ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq;
  fourvel<MET, T>(g, x[1], x[2], x[3], ucon, ucov, &gm);
  const T iut = g.alpha / gm;  // 1/u^t
  T rho = s.Dlab * iut;
  bvec_iut<MET, T>(g, ucon, ucov, iut, s.B[0], s.B[1], s.B[2], bcon, bcov, &bsq);
  T pg = (p.gam - 1.0) * x[0];
  T wb = rho + x[0] + pg + bsq, pt = pg + 0.5 * bsq;
  T Tc[4];
  Tc[0] = wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + rho * ucon[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) Tc[k] = wb * ucon[0] * ucov[k] - bcon[0] * bcov[k];
  T Rt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Rt[k] = s.Rs[k] - (Tc[k] - s.Ts[k]);
  T Pr[4];
  r.negE = rad_invert<MET, T>(p, g, Rt, 2, Pr);
  T urc[4], urv[4], gr;
  fourvel<MET, T>(g, Pr[1], Pr[2], Pr[3], urc, urv, &gr);
  T G[4];
  // T = p_g / rho0 = (gamma-1) u_g u^t / (rho0 u^t)
  four_force_rad<MET, T>(p, rho, (p.gam - 1.0) * x[0] * ucon[0] * s.iDlab, s.kf, s.ks, ucon, ucov, urc,
                         urv, Pr[0], G);
#pragma unroll
  for (int k = 0; k < 4; ++k) r.Eg[k] = Tc[k] - s.Ts[k] - s.h * G[k];
  T eS = T(-1.0);
  if (s.entropy) {
    // Eq. source6: S u^t(x) - S* = h G_S, S u^t = rho0 u^t s_gas, G_S = -G_mu u^mu / T
    // (Eq. GS), T = p/rho0; the radiation keeps total conservation (Sec. 4.7).
    // The row carries the factor F_13 = T (Sec. 4.8), E_S = T (S u^t - S*) +
    // h G_mu u^mu, and its norm adds the gas energy row's to its own terms.
    const T Tg = (p.gam - 1.0) * x[0] / rho;
    const T Gu = G[0] * ucon[0] + G[1] * ucon[1] + G[2] * ucon[2] + G[3] * ucon[3];
    const T Su = s.Dlab * entropy_per_baryon<T>(p, rho, x[0]);
    r.Eg[0] = Tg * (Su - s.Sstar) + s.h * Gu;
    if (norm) {
      const T d0 = Tg * (fabs(Su) + fabs(s.Sstar)) + s.h * fabs(Gu) +
                   (fabs(Tc[0]) + fabs(s.Ts[0]) + s.h * fabs(G[0]));
      eS = d0 > 0.0 ? fabs(r.Eg[0]) / d0 : T(0.0);
    }
  }
  if (norm) {
    T e43 = (4.0 / 3.0) * Pr[0];
    T Rc[4];
    Rc[0] = e43 * urc[0] * urv[0] + Pr[0] * (1.0 / 3.0);
#pragma unroll
    for (int k = 1; k < 4; ++k) Rc[k] = e43 * urc[0] * urv[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) r.Er[k] = Rc[k] - s.Rs[k] + s.h * G[k];
    normalise<MET, T>(s, Tc, Rc, G, true, r, eS);
    r.ok = isfinite(r.eT);
  } else {
    r.ok = true;
  }
  if (st) {
    st->negE = r.negE;
    st->rho = rho;
    st->ug = x[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      st->Pr[k] = Pr[k];
      st->Rt_pre[k] = Rt[k];
    }
  }
}

__device__ __forceinline__ bool solve4(double A[4][4], double b[4], double z[4]) {
  double ipv[4];  // reciprocals of the pivots, reused by the back-substitution
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    double best = fabs(A[c][c]);
#pragma unroll
    for (int r = c + 1; r < 4; ++r)
      if (fabs(A[r][c]) > best) {
        best = fabs(A[r][c]);
        piv = r;
      }
    if (best == 0.0 || !isfinite(best)) return false;
    if (piv != c) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double t = A[c][j];
        A[c][j] = A[piv][j];
        A[piv][j] = t;
      }
      double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    const double ip = 1.0 / A[c][c];
    ipv[c] = ip;
#pragma unroll
    for (int r = c + 1; r < 4; ++r) {
      double f = A[r][c] * ip;
#pragma unroll
      for (int j = c; j < 4; ++j) A[r][j] -= f * A[c][j];
      b[r] -= f * b[c];
    }
  }
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    double sum = b[i];
#pragma unroll
    for (int j = i + 1; j < 4; ++j) sum -= A[i][j] * z[j];
    z[i] = sum * ipv[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (!isfinite(z[i])) return false;
  return true;
}

// Error history for the stalled-error checks: the errors of the four previous
// iterates, shifted every iteration (register-resident: no indexed array).
struct Hist {
  double t1, t2, t3, t4;  // e_T of iterates k-1 .. k-4
  double i2, i3, i4, i1;  // e_I of iterates k-2 .. k-4, k-1
  int rises;
};

__device__ __forceinline__ bool stalled(Hist& hs, int k, double eT, double eI) {
  bool stop = false;
  if (k > 5) {
    if (eT > hs.t1) {
      hs.rises++;
      if (hs.rises >= 5) stop = true;
    }
    double mT = (hs.t4 + hs.t3 + hs.t2) / 3.0;
    double mI = (hs.i4 + hs.i3 + hs.i2) / 3.0;
    if (eT > 0.5 * mT || eI > 0.5 * mI) stop = true;
  }
  hs.t4 = hs.t3;
  hs.t3 = hs.t2;
  hs.t2 = hs.t1;
  hs.t1 = eT;
  hs.i4 = hs.i3;
  hs.i3 = hs.i2;
  hs.i2 = hs.i1;
  hs.i1 = eI;
  return stop;
}

// State of a PMHD Newton iteration between two of its steps: everything the
// next step depends on, so that an iteration can stop after a number of
// steps and resume later (in another kernel) with the same arithmetic.
struct NewtonState {
  double x[4];
  double best_x[4];
  double best_eT;
  Hist hs;
  double eps;
  int k;      // index of the next iteration
  int steps;  // Newton steps taken
  int jac32;  // 1 while the FP32 tangent Jacobian is in use, 0 after a fall-back
};

__device__ __forceinline__ void newton_pmhd_init(const double x0[4], NewtonState& st) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    st.x[i] = x0[i];
    st.best_x[i] = x0[i];
  }
  st.hs = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, 0};
  st.best_eT = HUGE_VAL;
  st.eps = 1e-8;
  st.k = 0;
  st.steps = 0;
  st.jac32 = 1;
}

// Finite-difference PMHD Jacobian (one-sided, the paper's numerical
// Jacobian): column j from the error at x + dj e_j, dj = eps |u_g| for j = 0
// and eps max(1, |u~|)/sqrt(g_jj) for the velocities.
template <int MET>
__device__ __forceinline__ void pmhd_jacobian_fd(const DevParams& p, const ImpSys<MET>& s, const double x[4],
                                                 const ImpRes& r, double eps, double J[4][4]) {
  double umag = fmax(1.0, sqrt(s.g.sq3(x[1], x[2], x[3])));
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    double dj = (j == 0) ? eps * fabs(x[0]) : eps * umag / sqrt(s.g.gdd(j));
    double xp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xp[i] = x[i] + (i == j ? dj : 0.0);
    ImpRes rp;
    pmhd_res<MET>(p, s, xp, rp, nullptr, false);
    double id = 1.0 / dj;
    // column j of J, written through compile-time indices
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (c == j) J[i][c] = (rp.Eg[i] - r.Eg[i]) * id;
  }
}

// Newton step dx = J^-1 E at x: the FP32 tangent Jacobian while *jac32, else
// (or when it is not finite or singular, which clears *jac32) the
// finite-difference one.  Returns false if no Jacobian could be solved.
template <int MET>
__device__ __forceinline__ bool pmhd_newton_dx(const DevParams& p, const ImpSys<MET>& s, const double x[4],
                                               const ImpRes& r, const double Rt[4], double eps, int* jac32,
                                               double dx[4], TanStage& ts) {
  if (*jac32) {
    double J[4][4];
    double E[4] = {r.Eg[0], r.Eg[1], r.Eg[2], r.Eg[3]};
    if (pmhd_jacobian_fp32<MET>(p, s, ts, x, Rt, J) && solve4(J, E, dx)) return true;
    *jac32 = 0;
  }
  double J[4][4];
  pmhd_jacobian_fd<MET>(p, s, x, r, eps, J);
  double E[4] = {r.Eg[0], r.Eg[1], r.Eg[2], r.Eg[3]};
  if (s.cold) {  // the 3x3 momentum block; u_g's row and column become the identity
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      J[0][i] = i == 0 ? 1.0 : 0.0;
      J[i][0] = i == 0 ? 1.0 : 0.0;
    }
    E[0] = 0.0;
  }
  return solve4(J, E, dx);
}

// PMHD Newton iterations from the state st until a stopping rule ends the
// iteration (returns true) or the next iteration's index reaches kstop
// (returns false; st holds what the remaining iterations need).  best_x /
// best_eT hold the lowest-error iterate (best_eT = inf if no residual was
// finite).
template <int MET>
__device__ __forceinline__ bool newton_pmhd_run(const DevParams& p, const ImpSys<MET>& s, NewtonState& st, int kstop) {
  TanStage ts;
  for (;; ++st.k) {
    if (st.k >= kstop) return false;
    ImpRes r;
    ImpState ist;
    pmhd_res<MET>(p, s, st.x, r, &ist, true);
    if (!r.ok) break;
    if (r.eT < st.best_eT) {
      st.best_eT = r.eT;
#pragma unroll
      for (int i = 0; i < 4; ++i) st.best_x[i] = st.x[i];
    }
    if (r.eT < p.newton_tol) break;
    // a step with the FP32 Jacobian that raised e_T: finite differences for
    // the rest of the solve
    if (st.jac32 && r.eT > st.hs.t1) st.jac32 = 0;
    if (stalled(st.hs, st.k, r.eT, r.eI)) break;
    if (st.k >= p.newton_max) break;
    if (r.eI < 1e-9) st.eps = 1e-10;
    double dx[4];
    if (!pmhd_newton_dx<MET>(p, s, st.x, r, ist.Rt_pre, st.eps, &st.jac32, dx, ts)) break;
    double xn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xn[i] = st.x[i] - dx[i];
    if (xn[0] < 0.0) xn[0] = 0.5 * fabs(xn[0]);
    bool tiny = true;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (fabs(xn[i] - st.x[i]) > 10.0 * 2.220446049250313e-16 * fabs(st.x[i])) tiny = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) st.x[i] = xn[i];
    ++st.steps;
    if (tiny) {
      ImpRes rf;
      pmhd_res<MET>(p, s, st.x, rf, nullptr, true);
      if (rf.ok && rf.eT < st.best_eT) {
        st.best_eT = rf.eT;
#pragma unroll
        for (int i = 0; i < 4; ++i) st.best_x[i] = st.x[i];
      }
      break;
    }
  }
  return true;
}

// PMHD Newton from x0 to the end (the same iterations as newton_pmhd_run
// without a pause, in local variables).  Returns the number of Newton steps;
// best_x / best_eT hold the lowest-error iterate (best_eT = inf if no
// residual was finite).
template <int MET>
__device__ int newton_pmhd(const DevParams& p, const ImpSys<MET>& s, const double x0[4],
                           double best_x[4], double* best_eT, ImpState* best_st = nullptr) {
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  Hist hs = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, 0};
  *best_eT = HUGE_VAL;
  int steps = 0;
  double eps = 1e-8;
  int jac32 = (s.entropy || s.cold) ? 0 : 1;  // the FP32 tangents differentiate the energy system
  TanStage ts;
  for (int k = 0;; ++k) {
    ImpRes r;
    ImpState ist;
    pmhd_res<MET>(p, s, x, r, &ist, true);
    if (!r.ok) break;
    if (r.eT < *best_eT) {
      *best_eT = r.eT;
#pragma unroll
      for (int i = 0; i < 4; ++i) best_x[i] = x[i];
      if (best_st) *best_st = ist;
    }
    if (r.eT < p.newton_tol) break;
    // a step with the FP32 Jacobian that raised e_T: finite differences for
    // the rest of the solve
    if (jac32 && r.eT > hs.t1) jac32 = 0;
    if (stalled(hs, k, r.eT, r.eI)) break;
    if (k >= p.newton_max) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double dx[4];
    if (!pmhd_newton_dx<MET>(p, s, x, r, ist.Rt_pre, eps, &jac32, dx, ts)) break;
    double xn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - dx[i];
    if (xn[0] < 0.0) xn[0] = 0.5 * fabs(xn[0]);
    bool tiny = true;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (fabs(xn[i] - x[i]) > 10.0 * 2.220446049250313e-16 * fabs(x[i])) tiny = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      ImpRes rf;
      ImpState stf;
      pmhd_res<MET>(p, s, x, rf, best_st ? &stf : nullptr, true);
      if (rf.ok && rf.eT < *best_eT) {
        *best_eT = rf.eT;
#pragma unroll
        for (int i = 0; i < 4; ++i) best_x[i] = x[i];
        if (best_st) *best_st = stf;
      }
      break;
    }
  }
  return steps;
}

// One damped Newton step of the PMHD system on a subset of its unknowns
// (the staged scheme of Sec. 4.9-4.10): unknowns not in `mask` (bit j for x_j)
// and their error rows drop out (identity row and column, zero error); the
// Jacobian columns come from two-sided differences with the PMHD offsets;
// x_new = x - D J^-1 E.  Returns false if the system is singular.
template <int MET>
__device__ bool pmhd_damped_step(const DevParams& p, const ImpSys<MET>& s, const double x[4], const ImpRes& r,
                                 unsigned mask, double D, double eps, double xn[4]) {
  const double umag = fmax(1.0, sqrt(s.g.sq3(x[1], x[2], x[3])));
  double J[4][4], E[4];
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    if (!(mask >> j & 1u)) {
      for (int i = 0; i < 4; ++i) J[i][j] = J[j][i] = i == j ? 1.0 : 0.0;
      continue;
    }
    const double dj = (j == 0) ? eps * fabs(x[0]) : eps * umag / sqrt(s.g.gdd(j));
    double xp[4], xm[4];
    for (int i = 0; i < 4; ++i) xp[i] = xm[i] = x[i];
    xp[j] += dj;
    xm[j] -= dj;
    ImpRes rp, rm;
    pmhd_res<MET>(p, s, xp, rp, nullptr, false);
    pmhd_res<MET>(p, s, xm, rm, nullptr, false);
    for (int i = 0; i < 4; ++i)
      if (mask >> i & 1u) J[i][j] = (rp.Eg[i] - rm.Eg[i]) / (2.0 * dj);
  }
  for (int i = 0; i < 4; ++i) E[i] = (mask >> i & 1u) ? r.Eg[i] : 0.0;
  double dx[4];
  if (!solve4(J, E, dx)) return false;
  for (int i = 0; i < 4; ++i) xn[i] = x[i] - D * dx[i];
  return true;
}

// Staged PMHD (Sec. 4.10) for zones whose radiation is extremely
// sub-dominant, after the plain methods: stage 1, one momentum-only step
// (u_g held) damped by 1/2; stage 2, energy-only steps (velocities held), the
// first damped by 1/2, until the energy row's normalised error is below the
// tolerance, has risen five times, or newton_max steps; stage 3, the full 4D
// Newton, its first step damped by 1/4, at most 40 steps, with the stopping
// rules of the plain method.  Two-sided differences throughout.  u_g < 0
// after a step becomes |u_g|/2; the second such reset in stage 1 or 2 keeps
// the prior iterate and ends the stage.  best_x / best_eT: the lowest-e_T
// iterate of all stages (inf if no residual was finite).  Returns the steps.
template <int MET>
__device__ int newton_pmhd_staged(const DevParams& p, const ImpSys<MET>& s, const double x0[4], double best_x[4],
                                  double* best_eT) {
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  *best_eT = HUGE_VAL;
  int steps = 0;
  double eps = 1e-8;
  auto eval = [&](ImpRes& r) {
    pmhd_res<MET>(p, s, x, r, nullptr, true);
    if (r.ok && r.eT < *best_eT) {
      *best_eT = r.eT;
      for (int i = 0; i < 4; ++i) best_x[i] = x[i];
    }
    return r.ok;
  };
#pragma unroll 1
  for (int stage = 1; stage <= 2; ++stage) {
    const unsigned mask = stage == 1 ? 0xEu : 0x1u;
    const int max_steps = stage == 1 ? 1 : p.newton_max;
    int resets = 0, rises = 0;
    double prev = HUGE_VAL;
#pragma unroll 1
    for (int k = 0; k < max_steps; ++k) {
      ImpRes r;
      if (!eval(r)) return steps;
      if (stage == 2) {
        if (r.eg0 < p.newton_tol) break;
        if (r.eg0 >= prev && ++rises >= 5) break;
        prev = r.eg0;
      }
      if (r.eI < 1e-9) eps = 1e-10;
      double xn[4];
      if (!pmhd_damped_step<MET>(p, s, x, r, mask, k == 0 ? 0.5 : 1.0, eps, xn)) break;
      ++steps;
      if (xn[0] < 0.0) {
        if (++resets >= 2) break;
        xn[0] = 0.5 * fabs(xn[0]);
      }
      for (int i = 0; i < 4; ++i) x[i] = xn[i];
    }
  }
  Hist hs = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, 0};
#pragma unroll 1
  for (int k = 0;; ++k) {
    ImpRes r;
    if (!eval(r)) break;
    if (r.eT < p.newton_tol) break;
    if (stalled(hs, k, r.eT, r.eI)) break;
    if (k >= 40) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double xn[4];
    if (!pmhd_damped_step<MET>(p, s, x, r, 0xFu, k == 0 ? 0.25 : 1.0, eps, xn)) break;
    if (xn[0] < 0.0) xn[0] = 0.5 * fabs(xn[0]);
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (fabs(xn[i] - x[i]) > 10.0 * 2.220446049250313e-16 * fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      ImpRes rf;
      eval(rf);
      break;
    }
  }
  return steps;
}

// The entropy-based URAD and PRAD (Sec. 4.8: their error function takes the
// entropy row and the three radiation momentum rows; the energy rows drop):
// the entropy row E_S = T (S u^t(P) - S*) + h G_mu u^mu (Eq. source6 with
// G_S of Eq. GS, times F_13 = T) in place of the radiation energy row; returns
// its normalised error (its terms plus the gas energy row's norm, Tc0 and G0
// the iterate's T^t_t + rho0 u^t and G_t) for normalise.
template <int MET>
__device__ __forceinline__ double entropy_rad_row(const DevParams& p, const ImpSys<MET>& s, double rho, double ug,
                                                  const double ucon[4], const double G[4], double Tc0, ImpRes& r) {
  const double Tg = (p.gam - 1.0) * ug / rho;
  const double Gu = G[0] * ucon[0] + G[1] * ucon[1] + G[2] * ucon[2] + G[3] * ucon[3];
  const double Su = s.Dlab * entropy_per_baryon<double>(p, rho, ug);
  r.Er[0] = Tg * (Su - s.Sstar) + s.h * Gu;
  const double d0 = Tg * (fabs(Su) + fabs(s.Sstar)) + s.h * fabs(Gu) + (fabs(Tc0) + fabs(s.Ts[0]) + s.h * fabs(G[0]));
  return d0 > 0.0 ? fabs(r.Er[0]) / d0 : 0.0;
}

// The u_g guess from the conserved entropy (Sec. 4.10, the guess of the PMHD
// method): the specific entropy s = S* / (rho0 u^t)* (Urho = sqrt(-g) rho0 u^t
// of U*) at the density rho0 of the guess gives p = (rho0^(n+1) e^s)^(1/n) and
// u_g = p / (Gamma - 1); x[0] is left unchanged where S* is not finite or the
// result is not a positive number.
__device__ __forceinline__ void entropy_ug_guess(const DevParams& p, double Sst, double Urho, double rho,
                                                 double x[4]) {
  if (!isfinite(Sst) || Urho == 0.0) return;
  const double n = 1.0 / (p.gam - 1.0);
  const double pg = exp((Sst / Urho + (n + 1.0) * log(rho)) / n);
  if (isfinite(pg) && pg > 0.0) x[0] = pg / (p.gam - 1.0);
}

// URAD error function: iterate R^t_nu; gas from 1D_W inversion of
// T^t_nu = T*^t_nu - (x - R*^t_nu); radiation from the M1 inversion of x.
template <int MET>
__device__ __forceinline__ bool urad_res(const DevParams& p, const ImpSys<MET>& s, const double x[4],
                                         const double Pg[5], double tol_inv, ImpRes& r,
                                         double gas_out[5], double Pr[4], bool norm) {
  const auto& g = s.g;
  double Tt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Tt[k] = s.Ts[k] - (x[k] - s.Rs[k]);
  double Pg12[12];
  Pg12[UU] = Pg[1];
  Pg12[U1] = Pg[2];
  Pg12[U2] = Pg[3];
  Pg12[U3] = Pg[4];
  double T3[3] = {Tt[1], Tt[2], Tt[3]};
  if (gas_invert<MET>(p, g, s.Dlab, Tt[0], T3, s.B, Pg12, tol_inv, gas_out) != 0) {
    r.ok = false;
    return false;
  }
  r.negE = rad_invert<MET>(p, g, x, 2, Pr);
  double ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq;
  fourvel<MET, double>(g, gas_out[2], gas_out[3], gas_out[4], ucon, ucov, &gm);
  bvec<MET, double>(g, ucon, ucov, s.B[0], s.B[1], s.B[2], bcon, bcov, &bsq);
  double rho = gas_out[0], ug = gas_out[1];
  double pg = (p.gam - 1.0) * ug;
  double wb = rho + ug + pg + bsq, pt = pg + 0.5 * bsq;
  double Tc[4];
  Tc[0] = wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + rho * ucon[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) Tc[k] = wb * ucon[0] * ucov[k] - bcon[0] * bcov[k];
  double urc[4], urv[4], gr;
  fourvel<MET, double>(g, Pr[1], Pr[2], Pr[3], urc, urv, &gr);
  double e43 = (4.0 / 3.0) * Pr[0];
  double Rc[4];
  Rc[0] = e43 * urc[0] * urv[0] + Pr[0] * (1.0 / 3.0);
#pragma unroll
  for (int k = 1; k < 4; ++k) Rc[k] = e43 * urc[0] * urv[k];
  double G[4];
  four_force_rad<MET>(p, rho, (p.gam - 1.0) * ug / rho, s.kf, s.ks, ucon, ucov, urc, urv, Pr[0], G);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r.Eg[k] = Tc[k] - s.Ts[k] - s.h * G[k];
    r.Er[k] = Rc[k] - s.Rs[k] + s.h * G[k];
  }
  const double eSr = s.entropy ? entropy_rad_row<MET>(p, s, rho, ug, ucon, G, Tc[0], r) : -1.0;
  if (norm) {
    normalise<MET>(s, Tc, Rc, G, false, r, -1.0, eSr);
    r.ok = isfinite(r.eT);
  } else {
    r.ok = true;
  }
  return r.ok;
}

// PRAD error function: iterate the radiation primitives (Ebar, u~^i_rad);
// R^t_nu from them in closed form; gas from 1D_W inversion of
// T^t_nu = T*^t_nu - (R^t_nu - R*^t_nu) (Sec. 4.8).
template <int MET>
__device__ __forceinline__ bool prad_res(const DevParams& p, const ImpSys<MET>& s, const double x[4],
                                         const double Pg[5], double tol_inv, ImpRes& r,
                                         double gas_out[5], double Rx[4], bool norm) {
  const auto& g = s.g;
  double urc[4], urv[4], gr;
  fourvel<MET, double>(g, x[1], x[2], x[3], urc, urv, &gr);
  const double e43 = (4.0 / 3.0) * x[0];
  Rx[0] = e43 * urc[0] * urv[0] + x[0] * (1.0 / 3.0);
#pragma unroll
  for (int k = 1; k < 4; ++k) Rx[k] = e43 * urc[0] * urv[k];
  double Tt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Tt[k] = s.Ts[k] - (Rx[k] - s.Rs[k]);
  double Pg12[12];
  Pg12[UU] = Pg[1];
  Pg12[U1] = Pg[2];
  Pg12[U2] = Pg[3];
  Pg12[U3] = Pg[4];
  double T3[3] = {Tt[1], Tt[2], Tt[3]};
  if (gas_invert<MET>(p, g, s.Dlab, Tt[0], T3, s.B, Pg12, tol_inv, gas_out) != 0) {
    r.ok = false;
    return false;
  }
  r.negE = 0;
  double ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq;
  fourvel<MET, double>(g, gas_out[2], gas_out[3], gas_out[4], ucon, ucov, &gm);
  bvec<MET, double>(g, ucon, ucov, s.B[0], s.B[1], s.B[2], bcon, bcov, &bsq);
  double rho = gas_out[0], ug = gas_out[1];
  double pg = (p.gam - 1.0) * ug;
  double wb = rho + ug + pg + bsq, pt = pg + 0.5 * bsq;
  double Tc[4];
  Tc[0] = wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + rho * ucon[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) Tc[k] = wb * ucon[0] * ucov[k] - bcon[0] * bcov[k];
  double G[4];
  four_force_rad<MET>(p, rho, (p.gam - 1.0) * ug / rho, s.kf, s.ks, ucon, ucov, urc, urv, x[0], G);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r.Eg[k] = Tc[k] - s.Ts[k] - s.h * G[k];
    r.Er[k] = Rx[k] - s.Rs[k] + s.h * G[k];
  }
  const double eSr = s.entropy ? entropy_rad_row<MET>(p, s, rho, ug, ucon, G, Tc[0], r) : -1.0;
  if (norm) {
    normalise<MET>(s, Tc, Rx, G, false, r, -1.0, eSr);
    r.ok = isfinite(r.eT);
  } else {
    r.ok = true;
  }
  return r.ok;
}

// Radiation-side Newton iterations (Sec. 4.8-4.10).  URAD (PRAD = false)
// iterates x = R^t_nu with offsets eps |R^t_t| (times sqrt(g_jj) for j > 0);
// PRAD iterates x = (Ebar, u~^i_rad) with offsets eps |Ebar| and
// eps max(1, |u~_rad|) / sqrt(g_jj).  Both: one-sided Jacobian of the
// radiation rows, offsets retried x10 up to 0.3 on an inversion failure,
// tolerance 1e-9, at most 20 x 6 gas inversions; an inversion error at a new
// iterate backs the step up half-way, up to 20 times; after a step URAD
// reflects R^t_t > 0 and PRAD Ebar < 0 to half their size.  Pg (gas guess:
// rho, u_g, u~^i) is updated by every successful residual.  best_x / best_Pg
// / best_eT hold the best iterate.
template <int MET, bool PRAD>
__device__ int newton_rad(const DevParams& p, const ImpSys<MET>& s, const double x0[4], double Pg[5],
                          double best_x[4], double best_Pg[5], double* best_eT) {
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  double xprev[4] = {x0[0], x0[1], x0[2], x0[3]};
  bool have_prev = false;
  Hist hs = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, 0};
  *best_eT = HUGE_VAL;
  int steps = 0, ninv = 0;
  const int budget = 20 * 6;
  double eps = 1e-8;
  auto res = [&](const double* xx, double tol, ImpRes& rr, double* go, bool norm) {
    double aux[4];
    return PRAD ? prad_res<MET>(p, s, xx, Pg, tol, rr, go, aux, norm)
                : urad_res<MET>(p, s, xx, Pg, tol, rr, go, aux, norm);
  };
  for (int k = 0;; ++k) {
    ImpRes r;
    double go[5];
    bool ok = false;
#pragma unroll 1
    for (int back = 0;; ++back) {
      ++ninv;
      ok = res(x, 1e-13, r, go, true);
      if (ok || !have_prev || back >= 20 || ninv >= budget) break;
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = 0.5 * (x[i] + xprev[i]);
    }
    if (!ok) break;
#pragma unroll
    for (int i = 0; i < 5; ++i) Pg[i] = go[i];
    if (r.eT < *best_eT) {
      *best_eT = r.eT;
#pragma unroll
      for (int i = 0; i < 4; ++i) best_x[i] = x[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) best_Pg[i] = go[i];
    }
    if (r.eT < 1e-9) break;
    if (stalled(hs, k, r.eT, r.eI)) break;
    if (k >= p.newton_max || ninv >= budget) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double J[4][4];
    bool jok = true;
    const double umag = PRAD ? fmax(1.0, sqrt(fmax(s.g.sq3(x[1], x[2], x[3]), 0.0))) : 0.0;
#pragma unroll 1
    for (int j = 0; j < 4 && jok; ++j) {
      double scale;
      if (PRAD)
        scale = j == 0 ? fabs(x[0]) : umag / sqrt(s.g.gdd(j));
      else
        scale = fabs(x[0]) * (j == 0 ? 1.0 : sqrt(s.g.gdd(j)));
      bool done = false;
#pragma unroll 1
      for (double e = eps; e <= 0.3 && !done; e *= 10.0) {
        double dj = e * scale;
        if (dj == 0.0) break;
        double xp[4] = {x[0], x[1], x[2], x[3]};
        xp[j] += dj;
        ImpRes rp;
        double go2[5];
        ++ninv;
        if (res(xp, 1e-2 * e, rp, go2, false)) {
          double id = 1.0 / dj;
#pragma unroll
          for (int i = 0; i < 4; ++i) J[i][j] = (rp.Er[i] - r.Er[i]) * id;
          done = true;
        }
      }
      if (!done) jok = false;
    }
    if (!jok) break;
    double E[4] = {r.Er[0], r.Er[1], r.Er[2], r.Er[3]}, dx[4];
    if (!solve4(J, E, dx)) break;
    double xn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - dx[i];
    if (PRAD) {
      if (xn[0] < 0.0) xn[0] = 0.5 * fabs(xn[0]);
    } else {
      if (xn[0] > 0.0) xn[0] = -0.5 * fabs(xn[0]);
    }
    bool tiny = true;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (fabs(xn[i] - x[i]) > 10.0 * 2.220446049250313e-16 * fabs(x[i])) tiny = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xprev[i] = x[i];
      x[i] = xn[i];
    }
    have_prev = true;
    ++steps;
    if (tiny) {
      ImpRes rf;
      double go3[5];
      ++ninv;
      if (res(x, 1e-13, rf, go3, true) && rf.eT < *best_eT) {
        *best_eT = rf.eT;
#pragma unroll
        for (int i = 0; i < 4; ++i) best_x[i] = x[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) best_Pg[i] = go3[i];
      }
      break;
    }
  }
  return steps;
}

// Staged URAD (PRAD = false) or PRAD (Sec. 4.10), after the plain methods for
// extremely sub-dominant radiation: one momentum-only step damped by 1/2,
// energy-only steps (the first damped by 1/2) until the radiation energy
// row's normalised error is below 1e-9, has risen five times or newton_max
// steps, then the full 4D Newton with its first step damped by 1/4, at most
// 40 steps; the plain method's controls otherwise (one-sided columns retried
// x10 up to 0.3, half-step back-off on an inversion failure, tolerance 1e-9),
// with 40 x 6 gas inversions in all.  The energy unknown reflected to half
// its size when a step puts it on the wrong side; the second reflection in
// stage 1 or 2 keeps the prior iterate and ends the stage.
template <int MET, bool PRAD>
__device__ int newton_rad_staged(const DevParams& p, const ImpSys<MET>& s, const double x0[4], double Pg[5],
                                 double best_x[4], double best_Pg[5], double* best_eT) {
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  double xprev[4] = {x0[0], x0[1], x0[2], x0[3]};
  bool have_prev = false;
  *best_eT = HUGE_VAL;
  int steps = 0, ninv = 0;
  const int budget = 40 * 6;
  double eps = 1e-8;
  auto res = [&](const double* xx, double tol, ImpRes& rr, double* go, bool norm) {
    double aux[4];
    ++ninv;
    return PRAD ? prad_res<MET>(p, s, xx, Pg, tol, rr, go, aux, norm)
                : urad_res<MET>(p, s, xx, Pg, tol, rr, go, aux, norm);
  };
  auto eval = [&](ImpRes& r) {
    double go[5];
    bool ok = false;
#pragma unroll 1
    for (int back = 0;; ++back) {
      ok = res(x, 1e-13, r, go, true);
      if (ok || !have_prev || back >= 20 || ninv >= budget) break;
      for (int i = 0; i < 4; ++i) x[i] = 0.5 * (x[i] + xprev[i]);
    }
    if (!ok) return false;
    for (int i = 0; i < 5; ++i) Pg[i] = go[i];
    if (r.eT < *best_eT) {
      *best_eT = r.eT;
      for (int i = 0; i < 4; ++i) best_x[i] = x[i];
      for (int i = 0; i < 5; ++i) best_Pg[i] = go[i];
    }
    return true;
  };
  auto step = [&](const ImpRes& r, unsigned mask, double D, double xn[4]) {
    double J[4][4], E[4];
    const double umag = PRAD ? fmax(1.0, sqrt(fmax(s.g.sq3(x[1], x[2], x[3]), 0.0))) : 0.0;
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      if (!(mask >> j & 1u)) {
        for (int i = 0; i < 4; ++i) J[i][j] = J[j][i] = i == j ? 1.0 : 0.0;
        continue;
      }
      const double scale = PRAD ? (j == 0 ? fabs(x[0]) : umag / sqrt(s.g.gdd(j)))
                                : fabs(x[0]) * (j == 0 ? 1.0 : sqrt(s.g.gdd(j)));
      bool done = false;
#pragma unroll 1
      for (double e = eps; e <= 0.3 && !done; e *= 10.0) {
        const double dj = e * scale;
        if (dj == 0.0) break;
        double xp[4] = {x[0], x[1], x[2], x[3]};
        xp[j] += dj;
        ImpRes rp;
        double go2[5];
        if (res(xp, 1e-2 * e, rp, go2, false)) {
          for (int i = 0; i < 4; ++i)
            if (mask >> i & 1u) J[i][j] = (rp.Er[i] - r.Er[i]) / dj;
          done = true;
        }
      }
      if (!done) return false;
    }
    for (int i = 0; i < 4; ++i) E[i] = (mask >> i & 1u) ? r.Er[i] : 0.0;
    double dx[4];
    if (!solve4(J, E, dx)) return false;
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - D * dx[i];
    return true;
  };
  auto wrong_side = [](double v) { return PRAD ? v < 0.0 : v > 0.0; };
  auto reflect = [](double v) { return PRAD ? 0.5 * fabs(v) : -0.5 * fabs(v); };
#pragma unroll 1
  for (int stage = 1; stage <= 2; ++stage) {
    const unsigned mask = stage == 1 ? 0xEu : 0x1u;
    const int max_steps = stage == 1 ? 1 : p.newton_max;
    int resets = 0, rises = 0;
    double prev = HUGE_VAL;
#pragma unroll 1
    for (int k = 0; k < max_steps; ++k) {
      ImpRes r;
      if (!eval(r)) return steps;
      if (stage == 2) {
        if (r.er0 < 1e-9) break;
        if (r.er0 >= prev && ++rises >= 5) break;
        prev = r.er0;
      }
      if (ninv >= budget) return steps;
      if (r.eI < 1e-9) eps = 1e-10;
      double xn[4];
      if (!step(r, mask, k == 0 ? 0.5 : 1.0, xn)) break;
      ++steps;
      if (wrong_side(xn[0])) {
        if (++resets >= 2) break;
        xn[0] = reflect(xn[0]);
      }
      for (int i = 0; i < 4; ++i) {
        xprev[i] = x[i];
        x[i] = xn[i];
      }
      have_prev = true;
    }
  }
  Hist hs = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL, 0};
#pragma unroll 1
  for (int k = 0;; ++k) {
    ImpRes r;
    if (!eval(r)) break;
    if (r.eT < 1e-9) break;
    if (stalled(hs, k, r.eT, r.eI)) break;
    if (k >= 40 || ninv >= budget) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double xn[4];
    if (!step(r, 0xFu, k == 0 ? 0.25 : 1.0, xn)) break;
    if (wrong_side(xn[0])) xn[0] = reflect(xn[0]);
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (fabs(xn[i] - x[i]) > 10.0 * 2.220446049250313e-16 * fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) {
      xprev[i] = x[i];
      x[i] = xn[i];
    }
    have_prev = true;
    ++steps;
    if (tiny) {
      ImpRes rf;
      double go3[5];
      if (res(x, 1e-13, rf, go3, true) && rf.eT < *best_eT) {
        *best_eT = rf.eT;
        for (int i = 0; i < 4; ++i) best_x[i] = x[i];
        for (int i = 0; i < 5; ++i) best_Pg[i] = go3[i];
      }
      break;
    }
  }
  return steps;
}

template <int MET>
__device__ __forceinline__ int newton_urad(const DevParams& p, const ImpSys<MET>& s, const double x0[4],
                                           double Pg[5], double best_x[4], double best_Pg[5], double* best_eT) {
  return newton_rad<MET, false>(p, s, x0, Pg, best_x, best_Pg, best_eT);
}

template <int MET, typename T = double>
__device__ __forceinline__ void build_sys(const DevParams& p, const Geo<MET, T>& g, const T Us[12], double h,
                                          T kf, ImpSysT<MET, T>& s) {
  s.g = g;
  s.kf = kf;
  s.ks = T(p.kscale);
  T igd = 1.0 / g.gdet;
  s.Dlab = Us[0] * igd;
  s.iDlab = 1.0 / s.Dlab;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s.Ts[k] = Us[1 + k] * igd;
    s.Rs[k] = Us[8 + k] * igd;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) s.B[i] = Us[5 + i] * igd;
  s.h = T(h);
  // orthonormal (ZAMO) size of covariant spatial components:
  // sqrt(gamma^{kk}), gamma^{kk} = g^{kk} - (g^{tk})^2 / g^{tt} > 0 everywhere
  // on the slice, inside the horizon too
#pragma unroll
  for (int k = 1; k < 4; ++k) s.sgk[k - 1] = sqrt(g.Gdd(k) - g.Gt(k) * g.Gt(k) / g.Gtt());
  s.entropy = false;
  s.cold = false;
  s.Sstar = T(0.0);
  (void)p;
}

}  // namespace hr
