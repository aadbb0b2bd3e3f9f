// HARMRAD oracle, implicit four-force solve -- TEST INFRASTRUCTURE ONLY.
//
// Restates Sec. 4.7-4.11 of McKinney et al. (2014): the energy-momentum
// equations T^t_nu(i+1) - T^t_nu(i) = h G_nu(i+1) (Eq. source3) with
// rho0 u^t and B fixed, solved by a 4D Newton-Raphson (Eq. newton) with a
// finite-difference Jacobian, first iterating the gas primitives (PMHD), then,
// if the error is not acceptable, the radiation conserved quantities (URAD),
// then the radiation primitives (PRAD); URAD first where the radiation is
// extremely sub-dominant (Sec. 4.10).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "oracle_internal.h"

namespace orc {

namespace {

struct Sys {
  const orc_params* p;
  const Geom* G;
  double Dlab;      // rho0 u^t (fixed)
  double Tstar[4];  // explicit T^t_nu with the rest-mass flux added to the t row
  double Rstar[4];  // explicit R^t_nu
  double B[3];      // lab field (fixed)
  double h;         // b_s dt
  bool entropy;     // solve the entropy equation in place of the gas energy row
  double Sstar;     // explicit S u^t (entropy density times u^t)
  bool cold;        // cold MHD: u_g held, momentum rows only (Sec. 4.11)
};

struct Res {
  double Eg[4], Er[4];  // gas and radiation error functions
  double eg[4], er[4];  // normalised per row
  double eT, eI;
  int negE;
  double Rt_pre[4];  // R^t_nu handed to the radiation inversion (pre-limiter)
  double P[NP];      // consistent primitives of this iterate
  bool ok;
};

// Normalised errors (Sec. 4.8): each row divided by the sum of the absolute
// values of the terms that make it up; the three spatial rows share one norm
// built in an orthonormal basis.  e_T takes, row by row, the larger of the gas
// and radiation errors; e_I uses the iterated rows only.  The orthonormal
// basis is the ZAMO frame: a covariant spatial component w_k has orthonormal
// size |w_k| sqrt(gamma^{kk}), gamma^{ij} = g^{ij} - g^{ti} g^{tj} / g^{tt}, the
// inverse metric of the t = const slice, positive also inside the horizon
// (where g^{rr} < 0).  The spatial norm also carries the terms of the energy
// row: momentum is bounded by energy, and a field at rest (all momentum terms
// zero) must not have its round-off divided by round-off.
double zamo_scale(const Geom& G, int k) {
  return std::sqrt(G.gcon[k][k] - G.gcon[0][k] * G.gcon[0][k] / G.gcon[0][0]);
}

void normalise(const Sys& s, const double Tc[4], const double Rc[4], const double Gc[4],
               bool iter_gas, Res& r) {
  const Geom& G = *s.G;
  double dg0 = std::fabs(Tc[0]) + std::fabs(s.Tstar[0]) + s.h * std::fabs(Gc[0]);
  double dr0 = std::fabs(Rc[0]) + std::fabs(s.Rstar[0]) + s.h * std::fabs(Gc[0]);
  double dgs = 0.0, drs = 0.0;
  for (int k = 1; k < 4; ++k) {
    double sk = zamo_scale(G, k);
    dgs += sk * (std::fabs(Tc[k]) + std::fabs(s.Tstar[k]) + s.h * std::fabs(Gc[k]));
    drs += sk * (std::fabs(Rc[k]) + std::fabs(s.Rstar[k]) + s.h * std::fabs(Gc[k]));
  }
  dgs += dg0;
  drs += dr0;
  r.eg[0] = dg0 > 0.0 ? std::fabs(r.Eg[0]) / dg0 : 0.0;
  r.er[0] = dr0 > 0.0 ? std::fabs(r.Er[0]) / dr0 : 0.0;
  for (int k = 1; k < 4; ++k) {
    double sk = zamo_scale(G, k);
    r.eg[k] = dgs > 0.0 ? std::fabs(r.Eg[k]) * sk / dgs : 0.0;
    r.er[k] = drs > 0.0 ? std::fabs(r.Er[k]) * sk / drs : 0.0;
  }
  if (r.negE) r.eg[0] = r.er[0] = 0.0;
  double sT = 0.0, sI = 0.0;
  for (int k = 0; k < 4; ++k) {
    sT += std::max(r.eg[k], r.er[k]);
    sI += iter_gas ? r.eg[k] : r.er[k];
  }
  r.eT = 0.25 * sT;
  r.eI = 0.25 * sI;
}

// T^t_nu in conserved form (rest-mass flux added to the t row) and R^t_nu.
void tt_row(const orc_params& p, const Geom& G, const double* P, double Tc[4], double Rc[4],
            FourVel* ug, double rho_u_t_out[1]) {
  double T[4][4], R[4][4], bcon[4], bcov[4], bsq;
  FourVel u, ur;
  gas_stress(p, G, P, T, u, bcon, bcov, &bsq);
  rad_stress(G, P, R, ur);
  double mt = P[RHO] * u.ucon[0];
  Tc[0] = T[0][0] + mt;
  for (int k = 1; k < 4; ++k) Tc[k] = T[0][k];
  for (int k = 0; k < 4; ++k) Rc[k] = R[0][k];
  if (ug) *ug = u;
  if (rho_u_t_out) rho_u_t_out[0] = mt;
}

// The entropy equation's error row at primitives P (gas four-velocity u,
// four-force Gc, gas energy row T^t_t + rho0 u^t = Tc[0]): Eq. source6,
// S u^t - S* - h G_S, times the factor F_13 = T = p/rho0 that Sec. 4.8 puts on
// the entropy row; since T G_S = -G_mu u^mu (Eq. GS) the row is
// E_S = T (S u^t - S*) + h G_mu u^mu.  Its normalised error (*e) divides
// |E_S| by the absolute values of its terms, T |S u^t| + T |S*| + h |G_mu u^mu|,
// plus the norm of the gas energy row |T^t_t + rho0 u^t| + |T*| + h |G_t| that
// Sec. 4.8 adds to it ("the energy norm").
double entropy_row(const Sys& s, const double* P, const FourVel& u, const double Gc[4], const double Tc[4],
                   double* e) {
  const orc_params& p = *s.p;
  const double Tg = (p.gam - 1.0) * P[UU] / P[RHO];
  const double Su = s.Dlab * entropy_per_baryon(p, P[RHO], P[UU]);
  double Gu = 0.0;
  for (int m = 0; m < 4; ++m) Gu += Gc[m] * u.ucon[m];
  const double E = Tg * (Su - s.Sstar) + s.h * Gu;
  const double dE = std::fabs(Tc[0]) + std::fabs(s.Tstar[0]) + s.h * std::fabs(Gc[0]);
  const double d = Tg * (std::fabs(Su) + std::fabs(s.Sstar)) + s.h * std::fabs(Gu) + dE;
  *e = d > 0.0 ? std::fabs(E) / d : 0.0;
  return E;
}

// PMHD error function: iterate (u_g, u~^i); rho0 = (rho0 u^t)/u^t; radiation
// from total energy-momentum conservation; then G_nu and E_q (Sec. 4.8).
void pmhd_res(const Sys& s, const double x[4], Res& r) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  double ut[3] = {x[1], x[2], x[3]};
  FourVel u;
  fourvel(G, ut, u);
  double P[NP];
  P[RHO] = s.Dlab / u.ucon[0];
  P[UU] = x[0];
  P[U1] = x[1];
  P[U2] = x[2];
  P[U3] = x[3];
  P[B1] = s.B[0];
  P[B2] = s.B[1];
  P[B3] = s.B[2];
  double T[4][4], bcon[4], bcov[4], bsq;
  gas_stress(p, G, P, T, u, bcon, bcov, &bsq);
  double Tc[4];
  Tc[0] = T[0][0] + P[RHO] * u.ucon[0];
  for (int k = 1; k < 4; ++k) Tc[k] = T[0][k];
  for (int k = 0; k < 4; ++k) r.Rt_pre[k] = s.Rstar[k] - (Tc[k] - s.Tstar[k]);
  double Pr[4];
  r.negE = rad_invert(p, G, r.Rt_pre, LIM_TYPE2, Pr);
  P[ER] = Pr[0];
  P[UR1] = Pr[1];
  P[UR2] = Pr[2];
  P[UR3] = Pr[3];
  double R[4][4];
  FourVel ur;
  rad_stress(G, P, R, ur);
  double Rc[4];
  for (int k = 0; k < 4; ++k) Rc[k] = R[0][k];
  double Gc[4];
  four_force(p, G, P[RHO], P[UU], u, R, Gc);
  for (int k = 0; k < 4; ++k) {
    r.Eg[k] = Tc[k] - s.Tstar[k] - s.h * Gc[k];
    r.Er[k] = Rc[k] - s.Rstar[k] + s.h * Gc[k];
  }
  normalise(s, Tc, Rc, Gc, true, r);
  if (s.entropy) {
    // Eq. source6 in place of the gas energy row: S u^t(x) - S* = h G_S with
    // S u^t = rho0 u^t s_gas, s_gas = log(p^n / rho0^(n+1)), n = 1/(Gamma-1)
    // (Sec. 2, Eq. S), and G_S = -G_mu u^mu / T, T = p/rho0 (Eq. GS).  The
    // radiation keeps total energy-momentum conservation (Sec. 4.7), so its
    // energy row only mirrors the gas energy equation that is not solved:
    // both energy rows leave e_T and e_I.  The row carries the factor
    // F_13 = T (Sec. 4.8) and is normalised with the gas energy row's norm
    // added (entropy_row).
    r.Eg[0] = entropy_row(s, P, u, Gc, Tc, &r.eg[0]);
    // a TYPE2 inversion that met a negative energy excludes the entropy term
    // from the error (Sec. 4.10)
    if (r.negE) r.eg[0] = 0.0;
    r.er[0] = 0.0;
    double sT = r.eg[0], sI = r.eg[0];
    for (int k = 1; k < 4; ++k) {
      sT += std::max(r.eg[k], r.er[k]);
      sI += r.eg[k];
    }
    r.eT = 0.25 * sT;
    r.eI = 0.25 * sI;
  }
  if (s.cold) {
    // cold MHD (Sec. 4.8, 4.11): energy and entropy errors are ignored, the
    // errors average the three momentum rows
    double sT = 0.0, sI = 0.0;
    for (int k = 1; k < 4; ++k) {
      sT += std::max(r.eg[k], r.er[k]);
      sI += r.eg[k];
    }
    r.eT = sT / 3.0;
    r.eI = sI / 3.0;
  }
  std::memcpy(r.P, P, sizeof(P));
  r.ok = std::isfinite(r.eT);
}

// The entropy equation's row for the radiation methods (Sec. 4.8: the
// entropy-based URAD and PRAD take the entropy row and the three radiation
// momentum rows as their error function; the energy rows are ignored): at the
// iterate's primitives P, the entropy row E_S of entropy_row replaces the
// radiation energy row of the Newton error vector, and e_T, e_I are formed as
// for the entropy PMHD with the radiation rows iterated.
void entropy_rad_rows(const Sys& s, const double* P, const FourVel& u, const double Gc[4], const double Tc[4],
                      Res& r) {
  double eS;
  r.Er[0] = entropy_row(s, P, u, Gc, Tc, &eS);
  // a TYPE2 inversion that met a negative energy excludes the entropy term
  // from the error (Sec. 4.10)
  if (r.negE) eS = 0.0;
  r.eg[0] = 0.0;
  r.er[0] = eS;
  double sT = eS, sI = eS;
  for (int k = 1; k < 4; ++k) {
    sT += std::max(r.eg[k], r.er[k]);
    sI += r.er[k];
  }
  r.eT = 0.25 * sT;
  r.eI = 0.25 * sI;
}

// URAD error function: iterate R^t_nu; gas from conservation through the
// 1D_W inversion; radiation from the M1 inversion; all conserved quantities
// recomputed from the primitives before forming E_q (Sec. 4.8).
bool urad_res(const Sys& s, const double x[4], const double* Pguess, double tol_inv, Res& r) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  double U[NP];
  double gd = G.gdet;
  U[0] = gd * s.Dlab;
  for (int k = 0; k < 4; ++k) U[1 + k] = gd * (s.Tstar[k] - (x[k] - s.Rstar[k]));
  for (int i = 0; i < 3; ++i) U[5 + i] = gd * s.B[i];
  for (int k = 0; k < 4; ++k) U[8 + k] = gd * x[k];
  double P[NP];
  if (gas_invert(p, G, U, Pguess, tol_inv, P) != 0) {
    r.ok = false;
    return false;
  }
  for (int k = 0; k < 4; ++k) r.Rt_pre[k] = x[k];
  double Pr[4];
  r.negE = rad_invert(p, G, x, LIM_TYPE2, Pr);
  P[ER] = Pr[0];
  P[UR1] = Pr[1];
  P[UR2] = Pr[2];
  P[UR3] = Pr[3];
  double Tc[4], Rc[4];
  FourVel u;
  tt_row(p, G, P, Tc, Rc, &u, nullptr);
  double T_[4][4], R[4][4];
  FourVel ur;
  (void)T_;
  rad_stress(G, P, R, ur);
  double Gc[4];
  four_force(p, G, P[RHO], P[UU], u, R, Gc);
  for (int k = 0; k < 4; ++k) {
    r.Eg[k] = Tc[k] - s.Tstar[k] - s.h * Gc[k];
    r.Er[k] = Rc[k] - s.Rstar[k] + s.h * Gc[k];
  }
  normalise(s, Tc, Rc, Gc, false, r);
  if (s.entropy) entropy_rad_rows(s, P, u, Gc, Tc, r);
  std::memcpy(r.P, P, sizeof(P));
  r.ok = std::isfinite(r.eT);
  return r.ok;
}

// PRAD error function: iterate the radiation primitives (Ebar, u~^i_rad);
// radiation R^t_nu from them in closed form; gas from total energy-momentum
// conservation through the 1D_W inversion; all conserved quantities
// recomputed from the primitives before forming E_q (Sec. 4.8).
bool prad_res(const Sys& s, const double x[4], const double* Pguess, double tol_inv, Res& r) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  double P[NP];
  for (int q = 0; q < NP; ++q) P[q] = Pguess[q];
  P[ER] = x[0];
  P[UR1] = x[1];
  P[UR2] = x[2];
  P[UR3] = x[3];
  double R[4][4];
  FourVel ur;
  rad_stress(G, P, R, ur);
  double Rx[4];
  for (int k = 0; k < 4; ++k) Rx[k] = R[0][k];
  double gd = G.gdet;
  double U[NP];
  U[0] = gd * s.Dlab;
  for (int k = 0; k < 4; ++k) U[1 + k] = gd * (s.Tstar[k] - (Rx[k] - s.Rstar[k]));
  for (int i = 0; i < 3; ++i) U[5 + i] = gd * s.B[i];
  for (int k = 0; k < 4; ++k) U[8 + k] = gd * Rx[k];
  double Pg[NP];
  if (gas_invert(p, G, U, Pguess, tol_inv, Pg) != 0) {
    r.ok = false;
    return false;
  }
  for (int q = 0; q < ER; ++q) P[q] = Pg[q];
  for (int k = 0; k < 4; ++k) r.Rt_pre[k] = Rx[k];
  r.negE = 0;
  double Tc[4], Rc[4];
  FourVel u;
  tt_row(p, G, P, Tc, Rc, &u, nullptr);
  double Gc[4];
  four_force(p, G, P[RHO], P[UU], u, R, Gc);
  for (int k = 0; k < 4; ++k) {
    r.Eg[k] = Tc[k] - s.Tstar[k] - s.h * Gc[k];
    r.Er[k] = Rc[k] - s.Rstar[k] + s.h * Gc[k];
  }
  normalise(s, Tc, Rc, Gc, false, r);
  if (s.entropy) entropy_rad_rows(s, P, u, Gc, Tc, r);
  std::memcpy(r.P, P, sizeof(P));
  r.ok = std::isfinite(r.eT);
  return r.ok;
}

// Solve A z = b (4x4) by Gaussian elimination with partial pivoting.
bool solve4(double A[4][4], double b[4], double z[4]) {
  double M[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) M[i][j] = A[i][j];
    M[i][4] = b[i];
  }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0 || !std::isfinite(M[piv][c])) return false;
    if (piv != c)
      for (int j = 0; j < 5; ++j) std::swap(M[c][j], M[piv][j]);
    for (int r = c + 1; r < 4; ++r) {
      double f = M[r][c] / M[c][c];
      for (int j = c; j < 5; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 3; i >= 0; --i) {
    double s = M[i][4];
    for (int j = i + 1; j < 4; ++j) s -= M[i][j] * z[j];
    z[i] = s / M[i][i];
  }
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(z[i])) return false;
  return true;
}

// Stopping checks shared by both methods (Sec. 4.10): after the 5th step the
// error must have halved relative to the mean of the errors 4, 3 and 2 steps
// earlier, and may not have risen 5 times.
struct History {
  double eT[64], eI[64];
  int rises = 0;
};
bool stalled(History& hs, int k) {
  if (k >= 1 && k > 5 && hs.eT[k] > hs.eT[k - 1]) {
    hs.rises++;
    if (hs.rises >= 5) return true;
  }
  if (k > 5) {
    double mT = (hs.eT[k - 4] + hs.eT[k - 3] + hs.eT[k - 2]) / 3.0;
    double mI = (hs.eI[k - 4] + hs.eI[k - 3] + hs.eI[k - 2]) / 3.0;
    if (hs.eT[k] > 0.5 * mT || hs.eI[k] > 0.5 * mI) return true;
  }
  return false;
}

// PMHD Newton (Sec. 4.9-4.10): undamped, one-sided FD Jacobian (the paper
// takes two-sided differences for PMHD only in its staged scheme, which is not
// used here) with a normalised offset of 1e-8 (1e-10 once e_I < 1e-9),
// u_g < 0 reset to |u_g|/2.  The cold-MHD system iterates the three momentum
// unknowns only (the reduced 3D method of Sec. 4.9): u_g keeps its guess.
int newton_pmhd(const Sys& s, const double x0[4], Res& best) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  History hs;
  best.eT = HUGE_VAL;
  best.ok = false;
  int steps = 0;
  double eps = 1e-8;
  for (int k = 0;; ++k) {
    Res r;
    pmhd_res(s, x, r);
    if (r.ok && r.eT < best.eT) best = r;
    if (!r.ok) break;
    hs.eT[k] = r.eT;
    hs.eI[k] = r.eI;
    if (r.eT < p.newton_tol) break;
    if (stalled(hs, k)) break;
    if (k >= p.newton_max) break;
    if (r.eI < 1e-9) eps = 1e-10;
    // Jacobian dE_gas/dx by forward differences
    double usq = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) usq += G.gcov[i + 1][j + 1] * x[1 + i] * x[1 + j];
    double umag = std::max(1.0, std::sqrt(usq));
    double J[4][4];
    for (int j = 0; j < 4; ++j) {
      if (s.cold && j == 0) {
        for (int i = 0; i < 4; ++i) J[i][0] = i == 0 ? 1.0 : 0.0;
        continue;
      }
      double dj = (j == 0) ? eps * std::fabs(x[0]) : eps * umag / std::sqrt(G.gcov[j][j]);
      double xp[4];
      for (int i = 0; i < 4; ++i) xp[i] = x[i];
      xp[j] += dj;
      Res rp;
      pmhd_res(s, xp, rp);
      for (int i = 0; i < 4; ++i) J[i][j] = (rp.Eg[i] - r.Eg[i]) / dj;
    }
    double dx[4], E[4] = {r.Eg[0], r.Eg[1], r.Eg[2], r.Eg[3]};
    if (s.cold) {
      // the 3x3 momentum block: the u_g row and column become the identity
      for (int j = 1; j < 4; ++j) J[0][j] = 0.0;
      E[0] = 0.0;
    }
    if (!solve4(J, E, dx)) break;
    double xn[4];
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - dx[i];
    if (xn[0] < 0.0) xn[0] = 0.5 * std::fabs(xn[0]);
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (std::fabs(xn[i] - x[i]) > 10.0 * EPSM * std::fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      Res rf;
      pmhd_res(s, x, rf);
      if (rf.ok && rf.eT < best.eT) best = rf;
      break;
    }
  }
  return steps;
}

// One damped Newton step of the PMHD system on a subset of its unknowns
// (Sec. 4.9-4.10, the staged scheme): the unknowns not in `mask` (bit j for
// x_j) and their error rows drop out (identity row and column, zero error),
// the Jacobian columns come from two-sided differences with the PMHD
// offsets, and x_new = x - D J^-1 E.  Returns false if the system is
// singular.
bool pmhd_damped_step(const Sys& s, const double x[4], const Res& r, unsigned mask, double D, double eps,
                      double xn[4]) {
  const Geom& G = *s.G;
  double usq = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) usq += G.gcov[i + 1][j + 1] * x[1 + i] * x[1 + j];
  const double umag = std::max(1.0, std::sqrt(usq));
  double J[4][4], E[4];
  for (int j = 0; j < 4; ++j) {
    if (!(mask >> j & 1u)) {
      for (int i = 0; i < 4; ++i) J[i][j] = J[j][i] = i == j ? 1.0 : 0.0;
      continue;
    }
    const double dj = (j == 0) ? eps * std::fabs(x[0]) : eps * umag / std::sqrt(G.gcov[j][j]);
    double xp[4], xm[4];
    for (int i = 0; i < 4; ++i) xp[i] = xm[i] = x[i];
    xp[j] += dj;
    xm[j] -= dj;
    Res rp, rm;
    pmhd_res(s, xp, rp);
    pmhd_res(s, xm, rm);
    for (int i = 0; i < 4; ++i)
      if (mask >> i & 1u) J[i][j] = (rp.Eg[i] - rm.Eg[i]) / (2.0 * dj);
  }
  for (int i = 0; i < 4; ++i) E[i] = (mask >> i & 1u) ? r.Eg[i] : 0.0;
  double dx[4];
  if (!solve4(J, E, dx)) return false;
  for (int i = 0; i < 4; ++i) xn[i] = x[i] - D * dx[i];
  return true;
}

// Staged PMHD (Sec. 4.10), for zones whose radiation is extremely
// sub-dominant, after the plain methods: stage 1, one momentum-only step
// (u_g held) damped by D = 1/2; stage 2, energy-only steps (velocities held),
// the first damped by 1/2, until the energy row's normalised error is below
// the tolerance, stops falling, or newton_max steps; stage 3, the full 4D
// Newton, its first step damped by 1/4, at most 40 steps, with the stopping
// rules of the plain method.  Two-sided differences throughout.  A step that
// leaves u_g < 0 sets it to |u_g|/2; the second such reset in stage 1 or 2
// restores the prior iterate and ends the stage.  The lowest-e_T iterate of
// all stages is kept.
int newton_pmhd_staged(const Sys& s, const double x0[4], Res& best) {
  const orc_params& p = *s.p;
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  best.eT = HUGE_VAL;
  best.ok = false;
  int steps = 0;
  double eps = 1e-8;
  auto eval = [&](Res& r) {
    pmhd_res(s, x, r);
    if (r.ok && r.eT < best.eT) best = r;
    return r.ok;
  };
  // stages 1 and 2
  for (int stage = 1; stage <= 2; ++stage) {
    const unsigned mask = stage == 1 ? 0xEu : 0x1u;
    const int max_steps = stage == 1 ? 1 : p.newton_max;
    int resets = 0, rises = 0;
    double prev = HUGE_VAL;
    for (int k = 0; k < max_steps; ++k) {
      Res r;
      if (!eval(r)) return steps;
      if (stage == 2) {
        if (r.eg[0] < p.newton_tol) break;
        if (r.eg[0] >= prev && ++rises >= 5) break;
        prev = r.eg[0];
      }
      if (r.eI < 1e-9) eps = 1e-10;
      double xn[4];
      if (!pmhd_damped_step(s, x, r, mask, k == 0 ? 0.5 : 1.0, eps, xn)) break;
      ++steps;
      if (xn[0] < 0.0) {
        if (++resets >= 2) break;  // hold the prior iterate, next stage
        xn[0] = 0.5 * std::fabs(xn[0]);
      }
      for (int i = 0; i < 4; ++i) x[i] = xn[i];
    }
  }
  // stage 3: full 4D
  History hs;
  for (int k = 0;; ++k) {
    Res r;
    if (!eval(r)) break;
    hs.eT[k] = r.eT;
    hs.eI[k] = r.eI;
    if (r.eT < p.newton_tol) break;
    if (stalled(hs, k)) break;
    if (k >= 40) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double xn[4];
    if (!pmhd_damped_step(s, x, r, 0xFu, k == 0 ? 0.25 : 1.0, eps, xn)) break;
    if (xn[0] < 0.0) xn[0] = 0.5 * std::fabs(xn[0]);
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (std::fabs(xn[i] - x[i]) > 10.0 * EPSM * std::fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      Res rf;
      eval(rf);
      break;
    }
  }
  return steps;
}

// URAD Newton (Sec. 4.8-4.10): one-sided FD Jacobian, tolerance 1e-9, at most
// 20 x 6 gas inversions, inversion failures inside the Jacobian retried with
// larger offsets up to 0.3.
int newton_urad(const Sys& s, const double x0[4], const double* Pg0, Res& best) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  const double tol = 1e-9;
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  double Pg[NP];
  std::memcpy(Pg, Pg0, sizeof(Pg));
  History hs;
  best.eT = HUGE_VAL;
  best.ok = false;
  int steps = 0, ninv = 0;
  const int inv_budget = 20 * 6;
  double eps = 1e-8;
  double xprev[4];
  bool have_prev = false;
  for (int k = 0;; ++k) {
    Res r;
    // an inversion error at a new iterate backs the step up half-way, up to
    // 20 times (Sec. 4.10)
    bool ok = false;
    for (int back = 0;; ++back) {
      ++ninv;
      ok = urad_res(s, x, Pg, 1e-13, r);
      if (ok || !have_prev || back >= 20 || ninv >= inv_budget) break;
      for (int i = 0; i < 4; ++i) x[i] = 0.5 * (x[i] + xprev[i]);
    }
    if (!ok) break;
    std::memcpy(Pg, r.P, sizeof(Pg));
    if (r.eT < best.eT) best = r;
    hs.eT[k] = r.eT;
    hs.eI[k] = r.eI;
    if (r.eT < tol) break;
    if (stalled(hs, k)) break;
    if (k >= p.newton_max || ninv >= inv_budget) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double J[4][4];
    bool jok = true;
    for (int j = 0; j < 4 && jok; ++j) {
      double scale = std::fabs(x[0]) * (j == 0 ? 1.0 : std::sqrt(G.gcov[j][j]));
      bool done = false;
      for (double e = eps; e <= 0.3 && !done; e *= 10.0) {
        double dj = e * scale;
        if (dj == 0.0) break;
        double xp[4] = {x[0], x[1], x[2], x[3]};
        xp[j] += dj;
        Res rp;
        ++ninv;
        if (urad_res(s, xp, Pg, 1e-2 * e, rp)) {
          for (int i = 0; i < 4; ++i) J[i][j] = (rp.Er[i] - r.Er[i]) / dj;
          done = true;
        }
      }
      if (!done) jok = false;
    }
    if (!jok) break;
    double dx[4], E[4] = {r.Er[0], r.Er[1], r.Er[2], r.Er[3]};
    if (!solve4(J, E, dx)) break;
    double xn[4];
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - dx[i];
    // R^t_t must stay negative (positive lab energy): reflect to half its size.
    if (xn[0] > 0.0) xn[0] = -0.5 * std::fabs(xn[0]);
    for (int i = 0; i < 4; ++i) xprev[i] = x[i];
    have_prev = true;
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (std::fabs(xn[i] - x[i]) > 10.0 * EPSM * std::fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      Res rf;
      ++ninv;
      if (urad_res(s, x, Pg, 1e-13, rf) && rf.eT < best.eT) best = rf;
      break;
    }
  }
  return steps;
}

// PRAD Newton (Sec. 4.8-4.10): iterate the radiation primitives (Ebar,
// u~^i_rad) with the URAD controls (one-sided Jacobian retried x10 up to 0.3
// on an inversion failure, tolerance 1e-9, 20 x 6 gas inversions, half-step
// back-off); offsets eps |Ebar| and eps max(1, |u~_rad|) / sqrt(g_jj) (the
// PMHD form for velocities); Ebar < 0 after a step -> |Ebar| / 2.
int newton_prad(const Sys& s, const double x0[4], const double* Pg0, Res& best) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  const double tol = 1e-9;
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  double Pg[NP];
  std::memcpy(Pg, Pg0, sizeof(Pg));
  History hs;
  best.eT = HUGE_VAL;
  best.ok = false;
  int steps = 0, ninv = 0;
  const int inv_budget = 20 * 6;
  double eps = 1e-8;
  double xprev[4];
  bool have_prev = false;
  for (int k = 0;; ++k) {
    Res r;
    // an inversion error at a new iterate backs the step up half-way, up to
    // 20 times (Sec. 4.10)
    bool ok = false;
    for (int back = 0;; ++back) {
      ++ninv;
      ok = prad_res(s, x, Pg, 1e-13, r);
      if (ok || !have_prev || back >= 20 || ninv >= inv_budget) break;
      for (int i = 0; i < 4; ++i) x[i] = 0.5 * (x[i] + xprev[i]);
    }
    if (!ok) break;
    std::memcpy(Pg, r.P, sizeof(Pg));
    if (r.eT < best.eT) best = r;
    hs.eT[k] = r.eT;
    hs.eI[k] = r.eI;
    if (r.eT < tol) break;
    if (stalled(hs, k)) break;
    if (k >= p.newton_max || ninv >= inv_budget) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double J[4][4];
    bool jok = true;
    for (int j = 0; j < 4 && jok; ++j) {
      double umag = 0.0;
      for (int a = 1; a < 4; ++a)
        for (int c = 1; c < 4; ++c) umag += G.gcov[a][c] * x[a] * x[c];
      umag = std::max(1.0, std::sqrt(std::max(umag, 0.0)));
      double scale = j == 0 ? std::fabs(x[0]) : umag / std::sqrt(G.gcov[j][j]);
      bool done = false;
      for (double e = eps; e <= 0.3 && !done; e *= 10.0) {
        double dj = e * scale;
        if (dj == 0.0) break;
        double xp[4] = {x[0], x[1], x[2], x[3]};
        xp[j] += dj;
        Res rp;
        ++ninv;
        if (prad_res(s, xp, Pg, 1e-2 * e, rp)) {
          for (int i = 0; i < 4; ++i) J[i][j] = (rp.Er[i] - r.Er[i]) / dj;
          done = true;
        }
      }
      if (!done) jok = false;
    }
    if (!jok) break;
    double dx[4], E[4] = {r.Er[0], r.Er[1], r.Er[2], r.Er[3]};
    if (!solve4(J, E, dx)) break;
    double xn[4];
    for (int i = 0; i < 4; ++i) xn[i] = x[i] - dx[i];
    // Ebar must stay positive: reflect to half its size (Sec. 4.10)
    if (xn[0] < 0.0) xn[0] = 0.5 * std::fabs(xn[0]);
    for (int i = 0; i < 4; ++i) xprev[i] = x[i];
    have_prev = true;
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (std::fabs(xn[i] - x[i]) > 10.0 * EPSM * std::fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      Res rf;
      ++ninv;
      if (prad_res(s, x, Pg, 1e-13, rf) && rf.eT < best.eT) best = rf;
      break;
    }
  }
  return steps;
}

// Staged URAD (prad = false) or PRAD (prad = true) (Sec. 4.10), after the
// plain methods for extremely sub-dominant radiation: the stages of the
// staged PMHD on the radiation unknowns -- one momentum-only step damped by
// 1/2, energy-only steps (the first damped by 1/2) until the radiation energy
// row's normalised error is below 1e-9, has risen five times or newton_max
// steps, then the full 4D Newton with its first step damped by 1/4, at most
// 40 steps -- with the plain method's controls: one-sided Jacobian columns
// retried with offsets x10 up to 0.3 on an inversion failure, an iterate
// whose inversion fails backed up half-way (up to 20 times), tolerance 1e-9,
// and 40 x 6 gas inversions in all (the staged budget).  A step that leaves
// the energy unknown on the wrong side (R^t_t > 0, Ebar < 0) reflects it to
// half its size; the second such reflection in stage 1 or 2 keeps the prior
// iterate and ends the stage.
int newton_rad_staged(const Sys& s, const double x0[4], const double* Pg0, bool prad, Res& best) {
  const orc_params& p = *s.p;
  const Geom& G = *s.G;
  const double tol = 1e-9;
  double x[4] = {x0[0], x0[1], x0[2], x0[3]};
  double Pg[NP];
  std::memcpy(Pg, Pg0, sizeof(Pg));
  best.eT = HUGE_VAL;
  best.ok = false;
  int steps = 0, ninv = 0;
  const int inv_budget = 40 * 6;
  double eps = 1e-8;
  double xprev[4];
  bool have_prev = false;
  auto res = [&](const double* xx, double tinv, Res& r) {
    ++ninv;
    return prad ? prad_res(s, xx, Pg, tinv, r) : urad_res(s, xx, Pg, tinv, r);
  };
  // the iterate's residual, backing the last step up half-way on an inversion failure
  auto eval = [&](Res& r) {
    bool ok = false;
    for (int back = 0;; ++back) {
      ok = res(x, 1e-13, r);
      if (ok || !have_prev || back >= 20 || ninv >= inv_budget) break;
      for (int i = 0; i < 4; ++i) x[i] = 0.5 * (x[i] + xprev[i]);
    }
    if (!ok) return false;
    std::memcpy(Pg, r.P, sizeof(Pg));
    if (r.eT < best.eT) best = r;
    return true;
  };
  // one damped step on the unknowns of mask
  auto step = [&](const Res& r, unsigned mask, double D, double xn[4]) {
    double J[4][4], E[4];
    for (int j = 0; j < 4; ++j) {
      if (!(mask >> j & 1u)) {
        for (int i = 0; i < 4; ++i) J[i][j] = J[j][i] = i == j ? 1.0 : 0.0;
        continue;
      }
      double scale;
      if (prad) {
        double umag = 0.0;
        for (int a = 1; a < 4; ++a)
          for (int c = 1; c < 4; ++c) umag += G.gcov[a][c] * x[a] * x[c];
        umag = std::max(1.0, std::sqrt(std::max(umag, 0.0)));
        scale = j == 0 ? std::fabs(x[0]) : umag / std::sqrt(G.gcov[j][j]);
      } else {
        scale = std::fabs(x[0]) * (j == 0 ? 1.0 : std::sqrt(G.gcov[j][j]));
      }
      bool done = false;
      for (double e = eps; e <= 0.3 && !done; e *= 10.0) {
        const double dj = e * scale;
        if (dj == 0.0) break;
        double xp[4] = {x[0], x[1], x[2], x[3]};
        xp[j] += dj;
        Res rp;
        if (res(xp, 1e-2 * e, rp)) {
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
  auto wrong_side = [&](double v) { return prad ? v < 0.0 : v > 0.0; };
  auto reflect = [&](double v) { return prad ? 0.5 * std::fabs(v) : -0.5 * std::fabs(v); };
  for (int stage = 1; stage <= 2; ++stage) {
    const unsigned mask = stage == 1 ? 0xEu : 0x1u;
    const int max_steps = stage == 1 ? 1 : p.newton_max;
    int resets = 0, rises = 0;
    double prev = HUGE_VAL;
    for (int k = 0; k < max_steps; ++k) {
      Res r;
      if (!eval(r)) return steps;
      if (stage == 2) {
        if (r.er[0] < tol) break;
        if (r.er[0] >= prev && ++rises >= 5) break;
        prev = r.er[0];
      }
      if (ninv >= inv_budget) return steps;
      if (r.eI < 1e-9) eps = 1e-10;
      double xn[4];
      if (!step(r, mask, k == 0 ? 0.5 : 1.0, xn)) break;
      ++steps;
      if (wrong_side(xn[0])) {
        if (++resets >= 2) break;
        xn[0] = reflect(xn[0]);
      }
      for (int i = 0; i < 4; ++i) xprev[i] = x[i];
      have_prev = true;
      for (int i = 0; i < 4; ++i) x[i] = xn[i];
    }
  }
  History hs;
  for (int k = 0;; ++k) {
    Res r;
    if (!eval(r)) break;
    hs.eT[k] = r.eT;
    hs.eI[k] = r.eI;
    if (r.eT < tol) break;
    if (stalled(hs, k)) break;
    if (k >= 40 || ninv >= inv_budget) break;
    if (r.eI < 1e-9) eps = 1e-10;
    double xn[4];
    if (!step(r, 0xFu, k == 0 ? 0.25 : 1.0, xn)) break;
    if (wrong_side(xn[0])) xn[0] = reflect(xn[0]);
    for (int i = 0; i < 4; ++i) xprev[i] = x[i];
    have_prev = true;
    bool tiny = true;
    for (int i = 0; i < 4; ++i)
      if (std::fabs(xn[i] - x[i]) > 10.0 * EPSM * std::fabs(x[i])) tiny = false;
    for (int i = 0; i < 4; ++i) x[i] = xn[i];
    ++steps;
    if (tiny) {
      Res rf;
      if (res(x, 1e-13, rf) && rf.eT < best.eT) best = rf;
      break;
    }
  }
  return steps;
}

void build_sys(const orc_params& p, const Geom& G, const double* Ustar, double h, Sys& s) {
  s.p = &p;
  s.G = &G;
  s.entropy = false;
  s.Sstar = 0.0;
  s.cold = false;
  double gd = G.gdet;
  s.Dlab = Ustar[0] / gd;
  for (int k = 0; k < 4; ++k) s.Tstar[k] = Ustar[1 + k] / gd;
  for (int k = 0; k < 4; ++k) s.Rstar[k] = Ustar[8 + k] / gd;
  for (int i = 0; i < 3; ++i) s.B[i] = Ustar[5 + i] / gd;
  s.h = h;
}

}  // namespace

// The u_g guess from the conserved entropy (Sec. 4.10, the guess of the PMHD
// method): the specific entropy s = S* / (rho0 u^t)* (Urho = sqrt(-g) rho0 u^t
// of U*) at the density rho0 of the guess gives p = (rho0^(n+1) e^s)^(1/n) and
// u_g = p / (Gamma - 1); x[0] is left unchanged where S* is not finite or
// the result is not a positive number.
void entropy_ug_guess(const orc_params& p, double Sstar, double Urho, double rho, double x[4]) {
  if (!std::isfinite(Sstar) || Urho == 0.0) return;
  const double n = 1.0 / (p.gam - 1.0);
  const double pg = std::exp((Sstar / Urho + (n + 1.0) * std::log(rho)) / n);
  if (std::isfinite(pg) && pg > 0.0) x[0] = pg / (p.gam - 1.0);
}

// Guess of the staged PMHD (Sec. 4.10): the gas of the lowest-error earlier
// solution if its e_T < 1e-4, else of P_s; u_g then from the specific
// entropy of U*, s_gas = S* / (rho0 u^t)*, at the density of P_s (where the
// explicit entropy S* is given).
void staged_guess(const orc_params& p, const Sys& s, const double* Ustar, const double* Sstar, const double* Ps,
                  const Res& best, double xs[4]) {
  const double* Pg = (best.ok && best.eT < 1e-4) ? best.P : Ps;
  for (int i = 0; i < 4; ++i) xs[i] = Pg[UU + i];
  if (Sstar) entropy_ug_guess(p, *Sstar, Ustar[RHO], Ps[RHO], xs);
  (void)s;
}

void method_zone(const orc_params& p, const Geom& G, const double* Ustar, const double* Sstar, const double* Ps,
                 double h, int method, double* Pout, double* eT, int* iters) {
  Sys s;
  build_sys(p, G, Ustar, h, s);
  Res b;
  if (method == 0) {
    double x0[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
    *iters = newton_pmhd(s, x0, b);
  } else if (method == 1) {
    double Tc[4], Rc[4];
    tt_row(p, G, Ps, Tc, Rc, nullptr, nullptr);
    *iters = newton_urad(s, Rc, Ps, b);
  } else if (method == 2) {
    double x0[4] = {Ps[ER], Ps[UR1], Ps[UR2], Ps[UR3]};
    *iters = newton_prad(s, x0, Ps, b);
  } else if (method == 3) {
    Res none;
    none.ok = false;
    double xs[4];
    staged_guess(p, s, Ustar, Sstar, Ps, none, xs);
    *iters = newton_pmhd_staged(s, xs, b);
  } else if (method == 4) {
    double Tc[4], Rc[4];
    tt_row(p, G, Ps, Tc, Rc, nullptr, nullptr);
    *iters = newton_rad_staged(s, Rc, Ps, false, b);
  } else if (method == 5) {
    double x0[4] = {Ps[ER], Ps[UR1], Ps[UR2], Ps[UR3]};
    *iters = newton_rad_staged(s, x0, Ps, true, b);
  } else {
    // the entropy-based PMHD, URAD, PRAD (Eq. source6 in place of the energy equation)
    Sys se = s;
    se.entropy = true;
    se.Sstar = Sstar ? *Sstar / G.gdet : 0.0;
    if (method == 6) {
      double x0[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
      *iters = newton_pmhd(se, x0, b);
    } else if (method == 7) {
      double Tc[4], Rc[4];
      tt_row(p, G, Ps, Tc, Rc, nullptr, nullptr);
      *iters = newton_urad(se, Rc, Ps, b);
    } else {
      double x0[4] = {Ps[ER], Ps[UR1], Ps[UR2], Ps[UR3]};
      *iters = newton_prad(se, x0, Ps, b);
    }
  }
  *eT = b.ok ? b.eT : HUGE_VAL;
  for (int q = 0; q < NP; ++q) Pout[q] = b.ok ? b.P[q] : Ps[q];
}

void pmhd_residual_public(const orc_params& p, const Geom& G, const double* Ustar, double h,
                          const double* xg, double* E4, double* eT, double* eI) {
  Sys s;
  build_sys(p, G, Ustar, h, s);
  Res r;
  pmhd_res(s, xg, r);
  for (int k = 0; k < 4; ++k) E4[k] = r.Eg[k];
  *eT = r.eT;
  *eI = r.eI;
}

// Sec. 4.10: the radiation is in the "extreme sub-dominant regime" when, on
// the energy row, its conserved value in U*, or its fluid-frame energy
// density, is below 10 eps_m of the gas's (u_g for the latter).  Then the
// round-off of the gas quantities from which PMHD recovers the radiation
// would swamp it, and URAD goes first.  (The paper also lists the relative
// change of the energy row over the explicit update; compared between gas and
// radiation it flags any zone whose radiation the update left unchanged, a
// uniform radiation field for one, whatever its size, so it is not used.)
bool radiation_subdominant(const Geom& G, const double* Ustar, const double* Ps) {
  const double tiny = 10.0 * 2.220446049250313e-16;
  if (std::fabs(Ustar[ER]) < tiny * std::fabs(Ustar[UU])) return true;
  // Ehat = R^{mu nu} u_mu u_nu = Ebar (4/3 gamma_rel^2 - 1/3), gamma_rel = -u_rad . u
  FourVel u, ur;
  double ut[3] = {Ps[U1], Ps[U2], Ps[U3]}, utr[3] = {Ps[UR1], Ps[UR2], Ps[UR3]};
  fourvel(G, ut, u);
  fourvel(G, utr, ur);
  double grel = 0.0;
  for (int m = 0; m < 4; ++m) grel -= ur.ucon[m] * u.ucov[m];
  double Ehat = Ps[ER] * ((4.0 / 3.0) * grel * grel - 1.0 / 3.0);
  return Ehat < tiny * Ps[UU];
}

// Sec. 4.11: the cold-MHD equations are tried only for a cold, momentum-
// dominated zone: u_g < 0.1 rho0 u~^i u~_i (guess primitives), and for both
// the gas t^t_mu = T^t_mu + rho0 u^t delta^t_mu and the radiation R^t_mu of
// U*, the time part of the covector's square, |t_t t^t| with
// t^t = g^{t mu} t_mu, below 0.1 of its spatial part |sum_i t_i t^i|.
bool cold_allowed(const Geom& G, const double* Ustar, const double* Ps) {
  double usq = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) usq += G.gcov[i + 1][j + 1] * Ps[U1 + i] * Ps[U1 + j];
  if (!(Ps[UU] < 0.1 * Ps[RHO] * usq)) return false;
  for (int w = 0; w < 2; ++w) {
    const double* c = Ustar + (w == 0 ? UU : ER);
    double t[4], tup[4];
    for (int m = 0; m < 4; ++m) t[m] = c[m] / G.gdet;
    for (int m = 0; m < 4; ++m) {
      tup[m] = 0.0;
      for (int n = 0; n < 4; ++n) tup[m] += G.gcon[m][n] * t[n];
    }
    double at = std::fabs(t[0] * tup[0]);
    double as = std::fabs(t[1] * tup[1] + t[2] * tup[2] + t[3] * tup[3]);
    if (!(at < 0.1 * as)) return false;
  }
  return true;
}

// Final primitives of a solve: the best iterate (B from U*), its radiation
// re-inverted with the BASIC limiter if the TYPE2 branch saw a negative
// energy; e_T > 1e-7 (or no finite iterate) is no solution: the back-up.
void finish_solution(const orc_params& p, const Geom& G, const Sys& s, const Res& best, const double* Ps,
                     double* Pout, orc_implicit_info* info, int method) {
  if (!best.ok) {
    for (int q = 0; q < NP; ++q) Pout[q] = Ps[q];
    for (int i = 0; i < 3; ++i) Pout[B1 + i] = s.B[i];
    info->e_T = HUGE_VAL;
    info->method = ORC_BACKUP;
    info->neg_erad = 0;
    return;
  }
  for (int q = 0; q < NP; ++q) Pout[q] = best.P[q];
  if (best.negE) {
    double Pr[4];
    rad_invert(p, G, best.Rt_pre, LIM_BASIC, Pr);
    Pout[ER] = Pr[0];
    Pout[UR1] = Pr[1];
    Pout[UR2] = Pr[2];
    Pout[UR3] = Pr[3];
  }
  info->e_T = best.eT;
  info->neg_erad = best.negE;
  info->method = (best.eT > 1e-7) ? ORC_BACKUP : method;
}

// After the entropy PMHD (bs), the entropy URAD and then the entropy PRAD
// while the best entropy solution has e_T >= 1e-9 (the energy methods'
// sequence, Sec. 4.11), each from the primitives of the best entropy solution
// if its e_T < 1e-4, else from P_s.  bs ends as the lowest-error entropy
// solution (*rad = 1 if URAD or PRAD gave it, else unchanged); returns the
// Newton steps.
int entropy_radiation_methods(const orc_params& p, const Geom& G, const Sys& se, const double* Ps, Res& bs,
                              int* rad) {
  int steps = 0;
  for (int prad = 0; prad < 2 && !(bs.ok && bs.eT < 1e-9); ++prad) {
    const double* Pg = (bs.ok && bs.eT < 1e-4) ? bs.P : Ps;
    double xr[4];
    if (prad) {
      for (int i = 0; i < 4; ++i) xr[i] = Pg[ER + i];
    } else {
      double Tc[4];
      tt_row(p, G, Pg, Tc, xr, nullptr, nullptr);
    }
    Res br;
    steps += prad ? newton_prad(se, xr, Pg, br) : newton_urad(se, xr, Pg, br);
    if (br.ok && (!bs.ok || br.eT < bs.eT)) {
      bs = br;
      *rad = 1;
    }
  }
  return steps;
}

// The cold-MHD back-up (Sec. 4.11): when cold_allowed, the PMHD method on
// the three momentum equations alone, u_g held at the guess x0's value; the
// gas and radiation energy equations are dropped, the radiation still takes
// total energy-momentum conservation.  Accepted at e_T <= 1e-7 (a retry
// method's solution, info->cold = 1); returns false otherwise.
bool try_cold(const orc_params& p, const Geom& G, const Sys& s, const double* Ustar, const double* Ps,
              const double x0[4], double* Pout, orc_implicit_info* info) {
  if (!cold_allowed(G, Ustar, Ps)) return false;
  Sys sc = s;
  sc.entropy = false;
  sc.cold = true;
  Res bc;
  info->iters_urad += newton_pmhd(sc, x0, bc);
  if (!(bc.ok && bc.eT <= 1e-7)) return false;
  finish_solution(p, G, sc, bc, Ps, Pout, info, ORC_OK_URAD);
  info->cold = 1;
  return true;
}

// Method sequence (Sec. 4.10-4.11): PMHD first, guessed from P_s or, where the
// cell is optically thin (tau < 2/3), from a gas inversion of U*; URAD if PMHD
// leaves e_T > 1e-9; PRAD if both do; the lowest-error solution is kept.  With
// the radiation extremely sub-dominant URAD goes first, from P_s, then PRAD,
// and PMHD (which would lose that radiation in the gas's round-off) is not
// tried; if they leave e_T >= 1e-9, the staged PMHD follows.  When no energy-based method reaches e_T <= 1e-7 and the explicit
// entropy S* is given (RK3), the entropy-based PMHD follows (Sec. 4.11); its
// solution counts as a retry method's.  e_T > 1e-7 after that marks the zone
// for the neighbour-average back-up.  A solution that hit the TYPE2
// negative-energy branch has its radiation re-inverted with the BASIC
// limiter.  With implicit_eq = 1 every zone solves the entropy equation.
// When neither the energy nor the entropy equation gives a solution, a cold,
// momentum-dominated zone (cold_allowed) tries the cold-MHD equations before
// the back-up; the grid step then replaces its u_g by the neighbour average.
void implicit_zone(const orc_params& p, const Geom& G, const double* Ustar, const double* Sstar,
                   const double* Ps, double h, double* Pout, orc_implicit_info* info, bool subdominant) {
  Sys s;
  build_sys(p, G, Ustar, h, s);
  info->entropy = 0;
  info->cold = 0;
  double x0[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
  double kabs, ksca;
  opacity(p, Ps[RHO], Ps[UU], &kabs, &ksca);
  double dl = 0.0;
  for (int d = 1; d <= 3; ++d)
    if (p.n[d - 1] > 1) dl = std::max(dl, std::sqrt(G.gcov[d][d]) * p.dx[d - 1]);
  double tau = (kabs + ksca) * dl;
  if (tau < 2.0 / 3.0) {
    double Pt[NP];
    if (gas_invert(p, G, Ustar, Ps, 1e-9, Pt) == 0) {
      x0[0] = Pt[UU];
      x0[1] = Pt[U1];
      x0[2] = Pt[U2];
      x0[3] = Pt[U3];
    }
  }
  Res best;
  int method;
  if (p.implicit_eq == 1 && Sstar) {
    // entropy equation for every zone (Eq. source6), PMHD iterates
    Sys se = s;
    se.entropy = true;
    se.Sstar = *Sstar / G.gdet;
    double xe[4] = {x0[0], x0[1], x0[2], x0[3]};
    entropy_ug_guess(p, *Sstar, Ustar[RHO], Ps[RHO], xe);
    info->iters_pmhd = newton_pmhd(se, xe, best);
    int rad = 0;
    info->iters_urad = entropy_radiation_methods(p, G, se, Ps, best, &rad);
    if (!(best.ok && best.eT <= 1e-7) && try_cold(p, G, s, Ustar, Ps, x0, Pout, info)) return;
    // the entropy PMHD is this mode's first method; URAD and PRAD are retries
    finish_solution(p, G, se, best, Ps, Pout, info, rad ? ORC_OK_URAD : ORC_OK_PMHD);
    info->entropy = best.ok && best.eT <= 1e-7;
    return;
  }
  if (!subdominant) {
    Res bp;
    info->iters_pmhd = newton_pmhd(s, x0, bp);
    info->iters_urad = 0;
    best = bp;
    method = ORC_OK_PMHD;
    if (!(bp.ok && bp.eT < 1e-9)) {
      const double* Pg = (bp.ok && bp.eT < 1e-4) ? bp.P : Ps;
      double Tc[4], Rc[4];
      tt_row(p, G, Pg, Tc, Rc, nullptr, nullptr);
      double xr[4] = {Rc[0], Rc[1], Rc[2], Rc[3]};
      Res br;
      info->iters_urad = newton_urad(s, xr, Pg, br);
      if (br.ok && (!best.ok || br.eT < best.eT)) {
        best = br;
        method = ORC_OK_URAD;
      }
    }
  } else {
    double Tc[4], Rc[4];
    tt_row(p, G, Ps, Tc, Rc, nullptr, nullptr);
    double xr[4] = {Rc[0], Rc[1], Rc[2], Rc[3]};
    Res br;
    info->iters_urad = newton_urad(s, xr, Ps, br);
    info->iters_pmhd = 0;
    best = br;
    method = ORC_OK_URAD;
  }
  if (!(best.ok && best.eT < 1e-9)) {
    // PRAD (Sec. 4.10), guessed from the best earlier solution if its
    // e_T < 1e-4, else from the optically thin limit (the M1 inversion of U*,
    // no source) where tau < 2/3, else from P_s; its outcome counts as URAD's
    // (a retry method solved the zone)
    double xq[4];
    const double* Pq = Ps;
    if (best.ok && best.eT < 1e-4) {
      Pq = best.P;
      for (int i = 0; i < 4; ++i) xq[i] = best.P[ER + i];
    } else if (tau < 2.0 / 3.0) {
      rad_invert(p, G, s.Rstar, LIM_TYPE2, xq);
    } else {
      for (int i = 0; i < 4; ++i) xq[i] = Ps[ER + i];
    }
    Res bq;
    info->iters_urad += newton_prad(s, xq, Pq, bq);
    if (bq.ok && (!best.ok || bq.eT < best.eT)) {
      best = bq;
      method = ORC_OK_URAD;
    }
  }
  if (subdominant && !(best.ok && best.eT < 1e-9)) {
    // the staged PMHD, URAD and PRAD (Sec. 4.10), for the extremely
    // sub-dominant radiation only, each from the lowest-error solution so far
    // if its e_T < 1e-4, else from P_s
    double xs[4];
    staged_guess(p, s, Ustar, Sstar, Ps, best, xs);
    Res bs;
    info->iters_urad += newton_pmhd_staged(s, xs, bs);
    if (bs.ok && (!best.ok || bs.eT < best.eT)) {
      best = bs;
      method = ORC_OK_URAD;
    }
    for (int prad = 0; prad < 2 && !(best.ok && best.eT < 1e-9); ++prad) {
      const double* Pg = (best.ok && best.eT < 1e-4) ? best.P : Ps;
      double xr[4];
      if (prad) {
        for (int i = 0; i < 4; ++i) xr[i] = Pg[ER + i];
      } else {
        double Tc[4];
        tt_row(p, G, Pg, Tc, xr, nullptr, nullptr);
      }
      Res br;
      info->iters_urad += newton_rad_staged(s, xr, Pg, prad == 1, br);
      if (br.ok && (!best.ok || br.eT < best.eT)) {
        best = br;
        method = ORC_OK_URAD;
      }
    }
  }
  if (Sstar && !(best.ok && best.eT <= 1e-7)) {
    // no energy-based solution: the entropy equation replaces the gas energy
    // equation (Sec. 4.7, Eq. source6; Sec. 4.11), PMHD iterates, the same
    // guess as the energy PMHD
    Sys se = s;
    se.entropy = true;
    se.Sstar = *Sstar / G.gdet;
    Res bs;
    double xe[4] = {x0[0], x0[1], x0[2], x0[3]};
    entropy_ug_guess(p, *Sstar, Ustar[RHO], Ps[RHO], xe);
    info->iters_urad += newton_pmhd(se, xe, bs);
    int rad = 0;
    info->iters_urad += entropy_radiation_methods(p, G, se, Ps, bs, &rad);
    if (bs.ok && bs.eT <= 1e-7) {
      finish_solution(p, G, se, bs, Ps, Pout, info, ORC_OK_URAD);
      info->entropy = 1;
      return;
    }
  }
  if (!(best.ok && best.eT <= 1e-7) && try_cold(p, G, s, Ustar, Ps, x0, Pout, info)) return;
  finish_solution(p, G, s, best, Ps, Pout, info, method);
}

}  // namespace orc
