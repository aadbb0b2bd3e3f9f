// HARMRAD oracle, point-wise physics -- TEST INFRASTRUCTURE ONLY.
//
// Plain FP64 restatement of the per-zone physics of McKinney et al. (2014):
// metric and connection, 4-vectors, stress tensors, conserved variables,
// fluxes, wave speeds, four-force, the M1 radiation inversion, the gas 1D_W
// inversion and the implicit four-force solve.  Written for clarity, not
// speed; nothing here is shared with the CUDA library.
#include "oracle_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace orc {

const double EPSM = std::numeric_limits<double>::epsilon();

// ---------------------------------------------------------------------------
// Forward-mode dual number with four partial derivatives, used only to take
// exact derivatives of the metric for the connection coefficients.
struct Dual {
  double v;
  double d[4];
  Dual(double x = 0.0) : v(x) { d[0] = d[1] = d[2] = d[3] = 0.0; }
};
static Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
static Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
static Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < 4; ++i) r.d[i] = -a.d[i];
  return r;
}
static Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
static Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < 4; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
static Dual sin(const Dual& a) {
  Dual r(std::sin(a.v));
  for (int i = 0; i < 4; ++i) r.d[i] = std::cos(a.v) * a.d[i];
  return r;
}
static Dual cos(const Dual& a) {
  Dual r(std::cos(a.v));
  for (int i = 0; i < 4; ++i) r.d[i] = -std::sin(a.v) * a.d[i];
  return r;
}
static Dual exp(const Dual& a) {
  Dual r(std::exp(a.v));
  for (int i = 0; i < 4; ++i) r.d[i] = r.v * a.d[i];
  return r;
}

// ---------------------------------------------------------------------------
// Metric (Sec. 2).  Kerr-Schild in (t, r, theta, phi) mapped from the uniform
// internal coordinates by r = R0 + exp(x1),
// theta = pi x2 + (1-h)/2 sin(2 pi x2), phi = 2 pi x3.
template <class S>
static void ks_msp_gcov(const orc_params& p, const S X[4], S g[4][4]) {
  using std::cos;
  using std::exp;
  using std::sin;
  const double pi = M_PI;
  const double a = p.a_spin, h = p.hslope;
  S ex = exp(X[1]);
  S r = S(p.R0) + ex;
  S th = S(pi) * X[2] + S(0.5 * (1.0 - h)) * sin(S(2.0 * pi) * X[2]);
  S J[4];
  J[0] = S(1.0);
  J[1] = ex;
  J[2] = S(pi) * (S(1.0) + S(1.0 - h) * cos(S(2.0 * pi) * X[2]));
  J[3] = S(2.0 * pi);
  S sth = sin(th), cth = cos(th);
  S s2 = sth * sth;
  S Sig = r * r + S(a * a) * cth * cth;
  S tr = S(2.0) * r / Sig;  // 2r/Sigma
  S ks[4][4];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) ks[m][n] = S(0.0);
  ks[0][0] = -(S(1.0) - tr);
  ks[0][1] = tr;
  ks[0][3] = -S(a) * tr * s2;
  ks[1][1] = S(1.0) + tr;
  ks[1][3] = -S(a) * s2 * (S(1.0) + tr);
  ks[2][2] = Sig;
  ks[3][3] = s2 * (Sig + S(a * a) * s2 * (S(1.0) + tr));
  ks[1][0] = ks[0][1];
  ks[3][0] = ks[0][3];
  ks[3][1] = ks[1][3];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) g[m][n] = ks[m][n] * J[m] * J[n];
}

// Inverse of a symmetric 4x4 matrix by Gauss-Jordan elimination with partial
// pivoting, after symmetric equilibration: with D = diag(1/sqrt(max_j
// |a_ij|)), g^-1 = D (D g D)^-1 D and det g = det(D g D) / det(D)^2.  In the
// internal coordinates the metric's entries span many decades (g_11 ~ r^2
// dr/dx1^2 ~ 1e12 at r = 1e6 against g_00 ~ 1), and eliminating on the raw
// entries leaves the small entries of the inverse (g^{t1} ~ 2/r^2) with a
// relative error of order 1e-16 times that spread; on the equilibrated
// matrix every entry of the inverse keeps round-off accuracy.  Returns the
// determinant.
static double invert4(const double g_in[4][4], double inv[4][4]) {
  double D[4];
  for (int i = 0; i < 4; ++i) {
    double m = 0.0;
    for (int j = 0; j < 4; ++j) m = std::max(m, std::fabs(g_in[i][j]));
    D[i] = m > 0.0 ? 1.0 / std::sqrt(m) : 1.0;
  }
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      a[i][j] = D[i] * g_in[i][j] * D[j];
      a[i][j + 4] = (i == j) ? 1.0 : 0.0;
    }
  double det = 1.0;
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < 8; ++j) std::swap(a[c][j], a[piv][j]);
      det = -det;
    }
    double d = a[c][c];
    det *= d;
    if (d == 0.0) continue;
    for (int j = 0; j < 8; ++j) a[c][j] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int j = 0; j < 8; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) inv[i][j] = D[i] * a[i][j + 4] * D[j];
  for (int i = 0; i < 4; ++i) det /= D[i] * D[i];
  return det;
}

void geom_at(const orc_params& p, double x1, double x2, double x3, Geom& G) {
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) G.gcov[m][n] = 0.0;
  G.x[0] = 0.0;
  G.x[1] = x1;
  G.x[2] = x2;
  G.x[3] = x3;
  if (p.metric == 0) {
    G.gcov[0][0] = -1.0;
    G.gcov[1][1] = G.gcov[2][2] = G.gcov[3][3] = 1.0;
    G.r = 1.0;
  } else {
    double X[4] = {0.0, x1, x2, x3};
    ks_msp_gcov<double>(p, X, G.gcov);
    G.r = p.R0 + std::exp(x1);
  }
  double det = invert4(G.gcov, G.gcon);
  G.gdet = std::sqrt(std::fabs(det));
  G.alpha = 1.0 / std::sqrt(-G.gcon[0][0]);
}

// Gamma^l_{m k} = 1/2 g^{l n} (d_k g_{n m} + d_m g_{n k} - d_n g_{m k}),
// derivatives taken exactly by forward-mode differentiation of the metric.
void connection_at(const orc_params& p, double x1, double x2, double x3,
                   double Gam[4][4][4]) {
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m)
      for (int k = 0; k < 4; ++k) Gam[l][m][k] = 0.0;
  if (p.metric == 0) return;
  Dual X[4];
  double xv[4] = {0.0, x1, x2, x3};
  for (int i = 0; i < 4; ++i) {
    X[i] = Dual(xv[i]);
    X[i].d[i] = 1.0;
  }
  Dual g[4][4];
  ks_msp_gcov<Dual>(p, X, g);
  double gv[4][4], gi[4][4], dg[4][4][4];  // dg[k][m][n] = d_k g_{mn}
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      gv[m][n] = g[m][n].v;
      for (int k = 0; k < 4; ++k) dg[k][m][n] = g[m][n].d[k];
    }
  invert4(gv, gi);
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m)
      for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int n = 0; n < 4; ++n)
          s += gi[l][n] * (dg[k][n][m] + dg[m][n][k] - dg[n][m][k]);
        Gam[l][m][k] = 0.5 * s;
      }
}

// ---------------------------------------------------------------------------
// 4-velocity from the ZAMO-relative u~^i (Sec. 2, Sec. 4.5):
// gamma = sqrt(1 + g_ij u~^i u~^j), u^t = gamma/alpha,
// u^i = u~^i + gamma eta^i with eta^i = -alpha g^{ti}.
void fourvel(const Geom& G, const double ut[3], FourVel& u) {
  double q = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q += G.gcov[i + 1][j + 1] * ut[i] * ut[j];
  u.gamma = std::sqrt(1.0 + q);
  u.ucon[0] = u.gamma / G.alpha;
  for (int i = 0; i < 3; ++i) u.ucon[i + 1] = ut[i] - u.gamma * G.alpha * G.gcon[0][i + 1];
  lower(G, u.ucon, u.ucov);
}

void lower(const Geom& G, const double vcon[4], double vcov[4]) {
  for (int m = 0; m < 4; ++m) {
    double s = 0.0;
    for (int n = 0; n < 4; ++n) s += G.gcov[m][n] * vcon[n];
    vcov[m] = s;
  }
}

// Fluid-frame field b^mu from the lab field B^i (Sec. 2):
// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t.
void bfield(const Geom& G, const FourVel& u, const double B[3], double bcon[4],
            double bcov[4], double* bsq) {
  double bt = 0.0;
  for (int i = 0; i < 3; ++i) bt += B[i] * u.ucov[i + 1];
  bcon[0] = bt;
  for (int i = 0; i < 3; ++i) bcon[i + 1] = (B[i] + bt * u.ucon[i + 1]) / u.ucon[0];
  lower(G, bcon, bcov);
  double s = 0.0;
  for (int m = 0; m < 4; ++m) s += bcon[m] * bcov[m];
  *bsq = s;
}

// Gas+EM stress tensor T^mu_nu (Eq. MAEM).
void gas_stress(const orc_params& p, const Geom& G, const double* P, double T[4][4],
                FourVel& u, double bcon[4], double bcov[4], double* bsq) {
  double ut[3] = {P[U1], P[U2], P[U3]};
  double B[3] = {P[B1], P[B2], P[B3]};
  fourvel(G, ut, u);
  bfield(G, u, B, bcon, bcov, bsq);
  double rho = P[RHO], ug = P[UU];
  double pg = (p.gam - 1.0) * ug;
  double w = rho + ug + pg + *bsq;
  double ptot = pg + 0.5 * (*bsq);
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n)
      T[m][n] = w * u.ucon[m] * u.ucov[n] + (m == n ? ptot : 0.0) - bcon[m] * bcov[n];
}

// M1 radiation stress tensor R^mu_nu = 4/3 Ebar u^mu u_nu + 1/3 Ebar delta (Eq. Rlab).
void rad_stress(const Geom& G, const double* P, double R[4][4], FourVel& ur) {
  double ut[3] = {P[UR1], P[UR2], P[UR3]};
  fourvel(G, ut, ur);
  double E = P[ER];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n)
      R[m][n] = (4.0 / 3.0) * E * ur.ucon[m] * ur.ucov[n] + (m == n ? E / 3.0 : 0.0);
}

// Absorption and scattering coefficients per unit proper length.  Mode 2 is a
// per-zone absorption field: the grid driver puts the zone's field value into
// kappa_abs0 of the parameters it passes down for that zone.
void opacity(const orc_params& p, double rho, double ug, double* kabs, double* ksca) {
  double T = (p.gam - 1.0) * ug / rho;
  if (p.opacity == 2) {
    *kabs = p.kappa_scale * p.kappa_abs0;
  } else if (p.opacity == 1) {
    double Tc = std::max(T, p.T_kappa_min);
    *kabs = p.kappa_scale * p.kappa_abs0 * rho * rho * std::pow(Tc, -3.5);
  } else {
    *kabs = p.kappa_scale * p.kappa_abs0 * rho;
  }
  *ksca = p.kappa_scale * p.kappa_es0 * rho;
}

// Covariant four-force G_nu (Eq. Gcov) with lambda = kappa_abs a_rad T^4.
void four_force(const orc_params& p, const Geom& G, double rho, double ug, const FourVel& u,
                const double R[4][4], double Gcov[4]) {
  double kabs, ksca;
  opacity(p, rho, ug, &kabs, &ksca);
  double T = (p.gam - 1.0) * ug / rho;
  double lam = kabs * p.a_rad * T * T * T * T;
  double Ru[4];
  for (int m = 0; m < 4; ++m) {
    double s = 0.0;
    for (int a = 0; a < 4; ++a) s += R[m][a] * u.ucon[a];
    Ru[m] = s;
  }
  double uRu = 0.0;
  for (int a = 0; a < 4; ++a) uRu += u.ucov[a] * Ru[a];
  double Gcon[4];
  for (int m = 0; m < 4; ++m)
    Gcon[m] = -(kabs * Ru[m] + lam * u.ucon[m]) - ksca * (Ru[m] + uRu * u.ucon[m]);
  lower(G, Gcon, Gcov);
}

// Conserved vector and geometric source (Sec. 4: U_q and SM_q).
void prim_to_cons(const orc_params& p, const Geom& G, const double Gam[4][4][4],
                  const double* P, double* U, double* SM) {
  double T[4][4], R[4][4], bcon[4], bcov[4], bsq;
  FourVel u, ur;
  gas_stress(p, G, P, T, u, bcon, bcov, &bsq);
  rad_stress(G, P, R, ur);
  double gd = G.gdet;
  double mflux = P[RHO] * u.ucon[0];
  U[0] = gd * mflux;
  U[1] = gd * (T[0][0] + mflux);
  for (int i = 0; i < 3; ++i) U[2 + i] = gd * T[0][i + 1];
  for (int i = 0; i < 3; ++i) U[5 + i] = gd * P[B1 + i];
  for (int n = 0; n < 4; ++n) U[8 + n] = gd * R[0][n];
  if (SM) {
    for (int q = 0; q < NP; ++q) SM[q] = 0.0;
    for (int n = 0; n < 4; ++n) {
      double sg = 0.0, sr = 0.0;
      for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) {
          sg += T[k][l] * Gam[l][n][k];
          sr += R[k][l] * Gam[l][n][k];
        }
      SM[1 + n] = gd * sg;
      SM[8 + n] = gd * sr;
    }
  }
}

// Lab-frame characteristic speeds along direction d for a fluid with
// 4-velocity u and rest-frame signal speed^2 c2 (Sec. 4.4): the covector
// k_mu = delta^d_mu - v delta^t_mu must satisfy (k.u)^2 = c2 (k.k + (k.u)^2).
void char_speeds(const Geom& G, const double ucon[4], double c2, int d, double* vmin,
                 double* vmax) {
  double Au = ucon[d], Bu = ucon[0];
  double AA = G.gcon[d][d], BB = G.gcon[0][0], AB = G.gcon[0][d];
  double qa = Bu * Bu - c2 * (BB + Bu * Bu);
  double qb = -2.0 * (Au * Bu - c2 * (AB + Au * Bu));
  double qc = Au * Au - c2 * (AA + Au * Au);
  double disc = qb * qb - 4.0 * qa * qc;
  if (disc < 0.0) disc = 0.0;
  double sd = std::sqrt(disc);
  double v1 = (-qb + sd) / (2.0 * qa);
  double v2 = (-qb - sd) / (2.0 * qa);
  *vmax = std::max(v1, v2);
  *vmin = std::min(v1, v2);
}

// Face physics for one reconstructed state: U, F^d and (gas, rad) speeds.
void face_state(const orc_params& p, const Geom& G, int d, const double* P, double* U,
                double* F, double sp[4]) {
  double T[4][4], R[4][4], bcon[4], bcov[4], bsq;
  FourVel u, ur;
  gas_stress(p, G, P, T, u, bcon, bcov, &bsq);
  rad_stress(G, P, R, ur);
  double gd = G.gdet;
  double mt = P[RHO] * u.ucon[0], md = P[RHO] * u.ucon[d];
  U[0] = gd * mt;
  U[1] = gd * (T[0][0] + mt);
  for (int i = 0; i < 3; ++i) U[2 + i] = gd * T[0][i + 1];
  for (int i = 0; i < 3; ++i) U[5 + i] = gd * P[B1 + i];
  for (int n = 0; n < 4; ++n) U[8 + n] = gd * R[0][n];
  F[0] = gd * md;
  F[1] = gd * (T[d][0] + md);
  for (int i = 0; i < 3; ++i) F[2 + i] = gd * T[d][i + 1];
  double vd = u.ucon[d] / u.ucon[0];
  for (int i = 0; i < 3; ++i) {
    double vi = u.ucon[i + 1] / u.ucon[0];
    F[5 + i] = gd * (P[B1 + i] * vd - P[B1 + d - 1] * vi);
  }
  F[5 + d - 1] = 0.0;
  for (int n = 0; n < 4; ++n) F[8 + n] = gd * R[d][n];
  // gas fast magnetosonic speed
  double rho = P[RHO], ug = P[UU], pg = (p.gam - 1.0) * ug;
  double w = rho + ug + pg;
  double cs2 = p.gam * pg / w;
  double va2 = bsq / (w + bsq);
  double cms2 = cs2 + va2 - cs2 * va2;
  if (cms2 > 1.0) cms2 = 1.0;
  if (cms2 < 0.0) cms2 = 0.0;
  char_speeds(G, u.ucon, cms2, d, &sp[0], &sp[1]);
  // radiation: c^2 = 1/3, limited by (4/(3 tau))^2 in optically thick cells
  double kabs, ksca;
  opacity(p, rho, ug, &kabs, &ksca);
  double tau = (kabs + ksca) * std::sqrt(G.gcov[d][d]) * p.dx[d - 1];
  double cr2 = 1.0 / 3.0;
  if (tau > 0.0) cr2 = std::min(cr2, (4.0 / (3.0 * tau)) * (4.0 / (3.0 * tau)));
  char_speeds(G, ur.ucon, cr2, d, &sp[2], &sp[3]);
}

// ---------------------------------------------------------------------------
// M1 inversion in the ZAMO frame (Sec. 4.6, Eqs. prsol, tvrsol, gammarvsy, ysol).
static double ymax_of_gamma(double gmax) {
  // Invert Eq. gammarvsy: with s = sqrt(4-3y), 4 G (s - 1) = s + 2, G = gamma^2.
  double G2 = gmax * gmax;
  double s = (4.0 * G2 + 2.0) / (4.0 * G2 - 1.0);
  return (4.0 - s * s) / 3.0;
}

int rad_invert(const orc_params& p, const Geom& G, const double Rt[4], int limiter,
               double out[4]) {
  double a = G.alpha;
  double Ucov[4];
  for (int m = 0; m < 4; ++m) Ucov[m] = a * Rt[m];
  double Erad = 0.0;  // -eta^mu U_mu = alpha^2 R^{tt}
  for (int m = 0; m < 4; ++m) Erad += a * G.gcon[0][m] * Ucov[m];
  double Ut[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int m = 0; m < 4; ++m) s += G.gcon[i + 1][m] * Ucov[m];
    Ut[i] = s + Erad * a * G.gcon[0][i + 1];  // U~^i = U^i - E eta^i
  }
  double Utsq = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Utsq += G.gcov[i + 1][j + 1] * Ut[i] * Ut[j];
  double ymax = ymax_of_gamma(p.gamma_rad_max);
  int negE = (Erad <= 0.0) ? 1 : 0;
  double y;
  if (limiter == LIM_BASIC) {
    if (Erad <= 0.0) {
      out[0] = 1e-300;
      out[1] = out[2] = out[3] = 0.0;
      return negE;
    }
    // y = 0 without momentum (Erad^2 may underflow for Erad near 1e-300)
    y = Utsq > 0.0 ? Utsq / (Erad * Erad) : 0.0;
    if (y < 0.0) {
      y = 0.0;
      Ut[0] = Ut[1] = Ut[2] = 0.0;
    }
    if (y > ymax) {
      double f = std::sqrt(ymax / y);
      for (int i = 0; i < 3; ++i) Ut[i] *= f;
      y = ymax;
    }
  } else {  // TYPE2: keep the momentum, raise the energy to reach y = ymax
    y = (Erad > 0.0) ? (Utsq > 0.0 ? Utsq / (Erad * Erad) : 0.0) : HUGE_VAL;
    if (Erad <= 0.0 || y > ymax) {
      Erad = 1e-150 + std::sqrt(Utsq / ymax);
      y = Utsq / (Erad * Erad);
    }
    if (y < 0.0) y = 0.0;
  }
  double gam2 = (2.0 - y + std::sqrt(4.0 - 3.0 * y)) / (4.0 * (1.0 - y));
  double prad = Erad / (4.0 * gam2 - 1.0);
  out[0] = 3.0 * prad;
  double gr = std::sqrt(gam2);
  for (int i = 0; i < 3; ++i) out[1 + i] = gr * Ut[i] / (4.0 * prad * gam2);
  return negE;
}

// Specific entropy of the gas (Sec. 2, Eq. S): s = log(p^n / rho0^(n+1))
// with n = 1/(Gamma - 1), p = (Gamma - 1) u_g; the entropy density is rho0 s.
double entropy_per_baryon(const orc_params& p, double rho, double ug) {
  const double n = 1.0 / (p.gam - 1.0);
  return n * std::log((p.gam - 1.0) * ug) - (n + 1.0) * std::log(rho);
}

// ---------------------------------------------------------------------------
// Gas 1D_W inversion (Sec. 4.5): Newton on the energy equation Eq. EMHD in the
// unknown W' = W - D, with v~^2 from Eq. vsqeq and v~^i from Eq. tveq.
int gas_invert(const orc_params& p, const Geom& G, const double* U, const double* Pg,
               double tol, double* out) {
  const double gd = G.gdet, a = G.alpha, gam = p.gam;
  double Dlab = U[0] / gd, taue = U[1] / gd;
  double Tt[3], B[3];
  for (int i = 0; i < 3; ++i) {
    Tt[i] = U[2 + i] / gd;
    B[i] = U[5 + i] / gd;
  }
  double Ttt = taue - Dlab;  // T^t_t
  double D = a * Dlab;
  // E' = E - D, E = alpha^2 T^{tt} = -T^t_t + alpha^2 g^{ti} T^t_i
  double Ep = -taue + (1.0 - a) * Dlab;
  for (int i = 0; i < 3; ++i) Ep += a * a * G.gcon[0][i + 1] * Tt[i];
  double E = Ep + D;
  double Qcov[4] = {a * Ttt, a * Tt[0], a * Tt[1], a * Tt[2]};
  double Qt[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int m = 0; m < 4; ++m) s += G.gcon[i + 1][m] * Qcov[m];
    Qt[i] = s + E * a * G.gcon[0][i + 1];
  }
  double Bz[3] = {a * B[0], a * B[1], a * B[2]};
  double QdB = 0.0, Bsq = 0.0, Qtsq = 0.0;
  for (int i = 0; i < 3; ++i) {
    QdB += Qcov[i + 1] * Bz[i];
    for (int j = 0; j < 3; ++j) {
      Bsq += G.gcov[i + 1][j + 1] * Bz[i] * Bz[j];
      Qtsq += G.gcov[i + 1][j + 1] * Qt[i] * Qt[j];
    }
  }
  if (!(D > 0.0) || !std::isfinite(E)) return 1;
  // initial guess from the guess primitives
  double ug0[3] = {Pg[U1], Pg[U2], Pg[U3]};
  double q0 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q0 += G.gcov[i + 1][j + 1] * ug0[i] * ug0[j];
  double gam0 = std::sqrt(1.0 + q0);
  double Wp = D * q0 / (1.0 + gam0) + gam * std::max(Pg[UU], 0.0) * gam0 * gam0;
  if (!(Wp > 0.0)) Wp = std::max(std::fabs(Ep), 1e-300);

  auto vsq_of = [&](double W) {
    return (Qtsq * W * W + QdB * QdB * (Bsq + 2.0 * W)) / ((Bsq + W) * (Bsq + W) * W * W);
  };
  auto resid = [&](double Wpv, double* f, double* df) -> bool {
    double W = Wpv + D;
    double vsq = vsq_of(W);
    if (!(vsq < 1.0) || !(W > 0.0)) return false;
    double g2 = 1.0 / (1.0 - vsq);
    double g = std::sqrt(g2);
    double usq = g2 * vsq;
    double chi = (Wpv - D * usq / (g + 1.0)) / g2;
    double pg = (gam - 1.0) / gam * chi;
    *f = Wpv - Ep - pg + 0.5 * Bsq * (1.0 + vsq) - QdB * QdB / (2.0 * W * W);
    double W3 = W * W * W, WB = W + Bsq;
    double dvsq = -2.0 / (W3 * WB * WB * WB) *
                  (QdB * QdB * (3.0 * W * WB + Bsq * Bsq) + Qtsq * W3);
    double dchi = (1.0 - vsq) - W * dvsq + 0.5 * D * g * dvsq;
    double dp = (gam - 1.0) / gam * dchi;
    *df = 1.0 - dp + 0.5 * Bsq * dvsq + QdB * QdB / W3;
    return true;
  };
  double f, df;
  // make the starting point admissible (v~^2 < 1)
  int guard = 0;
  while (!resid(Wp, &f, &df) && guard < 200) {
    Wp = 2.0 * Wp + 1e-300;
    ++guard;
  }
  if (guard >= 200) return 2;
  bool conv = false;
  for (int it = 0; it < 50; ++it) {
    if (!(df != 0.0) || !std::isfinite(f) || !std::isfinite(df)) return 3;
    double dW = -f / df;
    double Wn = Wp + dW;
    double fn, dfn;
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
    if (std::fabs(dW) <= tol * std::fabs(Wp)) {
      conv = true;
      break;
    }
  }
  if (!conv) return 5;
  double W = Wp + D;
  double vsq = vsq_of(W);
  double g2 = 1.0 / (1.0 - vsq);
  double g = std::sqrt(g2);
  double usq = g2 * vsq;
  double chi = (Wp - D * usq / (g + 1.0)) / g2;
  double rho = D / g;
  double ug = chi / gam;
  if (!(rho > 0.0) || !(ug > 0.0) || !std::isfinite(ug)) return 6;
  for (int q = 0; q < NP; ++q) out[q] = Pg[q];
  out[RHO] = rho;
  out[UU] = ug;
  for (int i = 0; i < 3; ++i) {
    double vt = (Qt[i] + QdB * Bz[i] / W) / (W + Bsq);
    out[U1 + i] = g * vt;
  }
  for (int i = 0; i < 3; ++i) out[B1 + i] = B[i];
  return 0;
}

}  // namespace orc
