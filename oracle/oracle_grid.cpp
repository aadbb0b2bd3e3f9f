// HARMRAD oracle, grid driver and C API -- TEST INFRASTRUCTURE ONLY.
//
// One full time step as restated from Sec. 4 of McKinney et al. (2014):
// the RK3 method with the same coefficients for the explicit and implicit
// parts (Sec. 4.1; the paper's runs), or one of the IMEX schemes IMEX2,
// IMEX2B, IMEX3 it prints in the same section; each sub-step runs the
// algorithm of Sec. 4.2 --
// ghost fill, U(P), geometric source, reconstruction (Sec. 4.3), face fluxes
// and wave speeds (Sec. 4.4), HLL/LAXF (Eqs. hll, lax), flux-CT EMFs, the
// update and the implicit solve with back-ups (Sec. 4.7-4.11).  Plain loops,
// FP64, one thread.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "oracle_internal.h"

namespace orc {

namespace {

const int NG = 4;  // ghost depth (PPM needs +-4 cells)

// Host threads for the zone and face loops: ORACLE_THREADS (default 1).  The
// loops are over independent zones and faces, so the result does not depend
// on the thread count.
int orc_threads() {
  const char* e = std::getenv("ORACLE_THREADS");
  int v = e ? std::atoi(e) : 1;
  return v > 0 ? v : 1;
}

struct Ctx {
  orc_params p;
  int n[3], ng[3], N[3];
  long ntot;
  std::vector<double> P;    // [NP][ntot], ghosts included
  std::vector<double> K;    // [ntot] absorption field (opacity mode 2 only), ghosts included
  std::vector<double> Un;   // [NP][ntot]
  std::vector<double> F[3]; // face fluxes [NP][ntot], face f of cell idx is its lower face
  std::vector<double> spd[3];  // per-face max signal speed
  std::vector<double> flat[3]; // [2][ntot] stored flattener (gas, rad), max over sub-steps
  std::vector<Geom> geo;       // cell-centre geometry, ghosts included
  std::vector<double> gam;     // cell-centre connection [ntot][64] (KS only)
  std::vector<unsigned char> status;  // active zones
  std::vector<int> iters;             // active zones
  std::vector<double> FS[3];  // face fluxes of the entropy S u^j [ntot] (RK3)
  std::vector<double> Sn;     // sqrt(-g) S u^t of the step's initial state [ntot]
  long long counts[7];
  std::vector<double> M[4];  // IMEX: implicit source of stage j, gas rows [4][ntot]
  // staggered field (emf = 1): sqrt(-g) B^d on the lower d-face of each cell
  // [ntot], its value at the start of the step, and the gas signal speeds
  // (v_max, v_min) of each d-face [2][ntot]
  std::vector<double> Bf[3], Bfn[3], gsp[3];
};

inline long idx(const Ctx& c, int i, int j, int k) {
  return ((long)(k + c.ng[2]) * c.N[1] + (j + c.ng[1])) * c.N[0] + (i + c.ng[0]);
}
inline long aidx(const Ctx& c, int i, int j, int k) {
  return ((long)k * c.n[1] + j) * c.n[0] + i;
}
// Parameters for the physics of cell t: in opacity mode 2 the cell's field
// value stands in for kappa_abs0.
inline orc_params cell_params(const Ctx& c, long t) {
  orc_params q = c.p;
  if (c.p.opacity == 2) q.kappa_abs0 = c.K[t];
  return q;
}
inline double xc(const Ctx& c, int d, int i) { return c.p.x0[d] + (i + 0.5) * c.p.dx[d]; }
inline double xf(const Ctx& c, int d, int i) { return c.p.x0[d] + i * c.p.dx[d]; }

// ---------------------------------------------------------------- boundaries
// Ghost fill in direction order 1, 2, 3 so that edges and corners are filled
// from already-filled data.  Periodic: wrap.  Outflow: copy the last active
// zone and clamp the normal velocities so nothing flows in from the ghost.
// Polar (direction 2 only): mirror across the axis, taking the zone on the
// opposite side in phi (shift n3/2) and negating the theta components.
// Fixed: the ghosts are left as set (orc_set_prims_with_ghosts).  The
// absorption field (opacity mode 2) is copied from the same source zone.
void fill_ghosts(Ctx& c, std::vector<double>& P) {
  for (int d = 0; d < 3; ++d) {
    if (c.n[d] == 1) continue;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      if (e < d) {
        lo[e] = -c.ng[e];
        hi[e] = c.n[e] + c.ng[e];
      } else {
        lo[e] = 0;
        hi[e] = c.n[e];
      }
    }
    for (int side = 0; side < 2; ++side) {
      int bc = c.p.bc[2 * d + side];
      if (bc == 4) continue;  // fixed: the ghosts keep the values they were given
      for (int g = 0; g < c.ng[d]; ++g) {
        int gi = side == 0 ? -1 - g : c.n[d] + g;
        int a0 = d == 0 ? 0 : lo[0], a1 = d == 0 ? 1 : hi[0];
        int b0 = d == 1 ? 0 : lo[1], b1 = d == 1 ? 1 : hi[1];
        int e0 = d == 2 ? 0 : lo[2], e1 = d == 2 ? 1 : hi[2];
        for (int k = e0; k < e1; ++k)
          for (int j = b0; j < b1; ++j)
            for (int i = a0; i < a1; ++i) {
              int dst[3] = {i, j, k}, src[3] = {i, j, k};
              dst[d] = gi;
              double sign_d = 1.0;
              int clamp = 0;
              if (bc == 0) {
                src[d] = side == 0 ? c.n[d] - 1 - g : g;
              } else if (bc == 1 || bc == 3) {
                src[d] = side == 0 ? 0 : c.n[d] - 1;
                clamp = bc == 3 ? 0 : (side == 0 ? -1 : 1);
              } else {
                src[d] = side == 0 ? g : c.n[d] - 1 - g;
                if (c.n[2] > 1) src[2] = (k + c.n[2] / 2) % c.n[2];
                sign_d = -1.0;
              }
              long s = idx(c, src[0], src[1], src[2]);
              long t = idx(c, dst[0], dst[1], dst[2]);
              for (int q = 0; q < NP; ++q) P[(long)q * c.ntot + t] = P[(long)q * c.ntot + s];
              if (!c.K.empty()) c.K[t] = c.K[s];
              if (sign_d < 0.0) {
                P[(long)(U1 + d) * c.ntot + t] *= -1.0;
                P[(long)(B1 + d) * c.ntot + t] *= -1.0;
                P[(long)(UR1 + d) * c.ntot + t] *= -1.0;
              }
              if (clamp != 0) {
                for (int q : {U1 + d, UR1 + d}) {
                  double& v = P[(long)q * c.ntot + t];
                  if (clamp < 0) v = std::min(v, 0.0);
                  else v = std::max(v, 0.0);
                }
              }
            }
      }
    }
  }
}

// ------------------------------------------------------------ reconstruction
// Monotonised-central slope.
double mc_slope(double qm, double q0, double qp) {
  double dl = q0 - qm, dr = qp - q0, dc = 0.5 * (qp - qm);
  if (dl * dr <= 0.0) return 0.0;
  double m = std::min(std::fabs(dc), std::min(2.0 * std::fabs(dl), 2.0 * std::fabs(dr)));
  return dc > 0.0 ? m : -m;
}

// PPM parabola of the centre cell of a 5-point stencil s[0..4] (Colella &
// Woodward 1984 without contact steepening), flattened by chi, then made
// monotone.  Returns the left and right edge values of the centre cell.
void ppm_cell(const double s[5], double chi, double* aL, double* aR) {
  double dm = mc_slope(s[0], s[1], s[2]);
  double d0 = mc_slope(s[1], s[2], s[3]);
  double dp = mc_slope(s[2], s[3], s[4]);
  double l = 0.5 * (s[1] + s[2]) - (d0 - dm) / 6.0;
  double r = 0.5 * (s[2] + s[3]) - (dp - d0) / 6.0;
  double q = s[2];
  l = (1.0 - chi) * l + chi * q;
  r = (1.0 - chi) * r + chi * q;
  if ((r - q) * (q - l) <= 0.0) {
    l = q;
    r = q;
  } else {
    double dd = r - l;
    double m6 = 6.0 * (q - 0.5 * (l + r));
    if (dd * m6 > dd * dd) l = 3.0 * q - 2.0 * r;
    else if (-dd * dd > dd * m6) r = 3.0 * q - 2.0 * l;
  }
  *aL = l;
  *aR = r;
}

// Shock flattener (Sec. 4.3): per cell, for GAS (gas pressure, sqrt(-g) u^d)
// and RAD (radiation pressure, sqrt(-g) u^d_rad); each pressure is blended
// toward the total with weight w = min(1, 2 tau) of the cell.
struct FlatIn {
  double pg, pr, vg, vr, w;
};
double ftilde(const FlatIn* c, int m, bool gas, double w) {
  auto pe = [&](int o) { return gas ? c[m + o].pg + w * c[m + o].pr : c[m + o].pr + w * c[m + o].pg; };
  auto ve = [&](int o) { return gas ? c[m + o].vg : c[m + o].vr; };
  double dp1 = pe(1) - pe(-1), dp2 = pe(2) - pe(-2);
  double dv = ve(1) - ve(-1);
  if (std::fabs(dp1) > 0.33 * std::min(pe(1), pe(-1)) && dv < 0.0) {
    double sp = dp2 != 0.0 ? dp1 / dp2 : 0.0;
    return std::max(0.0, std::min(1.0, 10.0 * (sp - 0.75)));
  }
  return 0.0;
}

// Flattener of cell m of the stencil array (needs m-3..m+3).
void flattener(const FlatIn* c, int m, double* fg, double* fr) {
  double g0 = ftilde(c, m, true, c[m].w), r0 = ftilde(c, m, false, c[m].w);
  double wg = c[m].w;
  double pg1 = c[m + 1].pg + wg * c[m + 1].pr, pgm = c[m - 1].pg + wg * c[m - 1].pr;
  double pr1 = c[m + 1].pr + wg * c[m + 1].pg, prm = c[m - 1].pr + wg * c[m - 1].pg;
  int sg = (pg1 - pgm) < 0.0 ? 1 : -1;
  int sr = (pr1 - prm) < 0.0 ? 1 : -1;
  double g = std::max(g0, ftilde(c, m + sg, true, c[m + sg].w));
  double r = std::max(r0, ftilde(c, m + sr, false, c[m + sr].w));
  double mx = std::max(g, r);
  *fg = (1.0 - wg) * g + wg * mx;
  *fr = (1.0 - wg) * r + wg * mx;
}


// Flux through one face of direction d (0-based) from its 8-cell stencil
// s[m] (cells f-4 .. f+3) with the stencil cells' geometry geo[m]; fg/fr
// return the flattener of the left (m = 3) and right (m = 4) cells.  When
// stored != nullptr the flattener is max-ed with (and written back to) the
// values of earlier sub-steps: stored[side][gas/rad].  K8 (opacity mode 2,
// else nullptr): the stencil cells' absorption field; a reconstructed face
// state takes the value of the cell it was reconstructed from.
void face_flux(const orc_params& p, int d, const double P8[8][NP], const Geom* geo[8], const Geom& Gf,
               const double* K8, double* stored[2][2], double F[NP], double* speed, double* FS = nullptr,
               double* gas_speeds = nullptr) {
  auto at = [&](int m) {
    orc_params q = p;
    if (K8) q.kappa_abs0 = K8[m];
    return q;
  };
  const bool wvar = p.metric == 1 && d != 1;
  auto weighted = [&](int q) { return wvar && ((q >= U1 && q <= B3) || (q >= UR1 && q <= UR3)); };
  double s[8][NP];
  FlatIn fin[8];
  for (int m = 0; m < 8; ++m) {
    const Geom& G = *geo[m];
    const double* Pm = P8[m];
    for (int q = 0; q < NP; ++q) s[m][q] = weighted(q) ? G.gdet * Pm[q] : Pm[q];
    double ut[3] = {Pm[U1], Pm[U2], Pm[U3]}, ur[3] = {Pm[UR1], Pm[UR2], Pm[UR3]};
    FourVel u, v;
    fourvel(G, ut, u);
    fourvel(G, ur, v);
    fin[m].pg = (p.gam - 1.0) * Pm[UU];
    fin[m].pr = Pm[ER] / 3.0;
    fin[m].vg = G.gdet * u.ucon[d + 1];
    fin[m].vr = G.gdet * v.ucon[d + 1];
    double ka, ks;
    opacity(at(m), Pm[RHO], Pm[UU], &ka, &ks);
    double tau = (ka + ks) * std::sqrt(G.gcov[d + 1][d + 1]) * p.dx[d];
    fin[m].w = std::min(1.0, 2.0 * tau);
  }
  double PL[NP], PR[NP];
  for (int side = 0; side < 2; ++side) {
    int m = side == 0 ? 3 : 4;  // cell f-1 (left state) or f (right state)
    double fg = 0.0, fr = 0.0;
    if (p.recon == 0) {
      flattener(fin, m, &fg, &fr);
      if (stored) {
        double& sg = *stored[side][0];
        double& sr = *stored[side][1];
        fg = std::max(fg, sg);
        fr = std::max(fr, sr);
        sg = fg;
        sr = fr;
      }
    }
    for (int q = 0; q < NP; ++q) {
      double aL, aR;
      if (p.recon == 0) {
        double st[5] = {s[m - 2][q], s[m - 1][q], s[m][q], s[m + 1][q], s[m + 2][q]};
        ppm_cell(st, q < ER ? fg : fr, &aL, &aR);
      } else {
        double dq = mc_slope(s[m - 1][q], s[m][q], s[m + 1][q]);
        aL = s[m][q] - 0.5 * dq;
        aR = s[m][q] + 0.5 * dq;
      }
      if (side == 0) PL[q] = aR;
      else PR[q] = aL;
    }
  }
  for (int q = 0; q < NP; ++q)
    if (weighted(q)) {
      PL[q] /= Gf.gdet;
      PR[q] /= Gf.gdet;
    }
  double UL[NP], UR[NP], FL[NP], FR[NP], sL[4], sR[4];
  face_state(at(3), Gf, d + 1, PL, UL, FL, sL);
  face_state(at(4), Gf, d + 1, PR, UR, FR, sR);
  double cmaxg = std::max(0.0, std::max(sL[1], sR[1]));
  double cming = -std::min(0.0, std::min(sL[0], sR[0]));
  double cmaxr = std::max(0.0, std::max(sL[3], sR[3]));
  double cminr = -std::min(0.0, std::min(sL[2], sR[2]));
  for (int q = 0; q < NP; ++q) {
    double cmx = q < ER ? cmaxg : cmaxr, cmn = q < ER ? cming : cminr;
    double fl;
    if (p.flux == 0) {
      double ctop = std::max(cmx, cmn);
      fl = 0.5 * (FL[q] + FR[q] - ctop * (UR[q] - UL[q]));
    } else {
      if (cmx + cmn > 0.0)
        fl = (cmn * FR[q] + cmx * FL[q] - cmn * cmx * (UR[q] - UL[q])) / (cmn + cmx);
      else
        fl = 0.5 * (FL[q] + FR[q]);
    }
    F[q] = fl;
  }
  *speed = std::max(std::max(cmaxg, cming), std::max(cmaxr, cminr));
  if (gas_speeds) {
    gas_speeds[0] = cmaxg;
    gas_speeds[1] = cming;
  }
  if (FS) {
    // entropy flux sqrt(-g) S u^d = s_gas F_rho and conserved s_gas U_rho of
    // each state (Sec. 4 list of U_q, F_q), with the gas signal speeds
    const double sL = entropy_per_baryon(at(3), PL[RHO], PL[UU]);
    const double sR = entropy_per_baryon(at(4), PR[RHO], PR[UU]);
    const double fL = sL * FL[RHO], fR = sR * FR[RHO], uL = sL * UL[RHO], uR = sR * UR[RHO];
    if (p.flux == 0) {
      *FS = 0.5 * (fL + fR - std::max(cmaxg, cming) * (uR - uL));
    } else if (cmaxg + cming > 0.0) {
      *FS = (cming * fR + cmaxg * fL - cming * cmaxg * (uR - uL)) / (cming + cmaxg);
    } else {
      *FS = 0.5 * (fL + fR);
    }
  }
}

// Face fluxes along direction d (0-based) for every face that the update or
// the flux-CT averaging needs; stores the per-face signal speed.  When
// use_stored is true the flattener is max-ed with (and written back to) the
// value stored from earlier sub-steps of this step.
void compute_fluxes(Ctx& c, int d, bool use_stored) {
  const orc_params& p = c.p;
  int lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    if (e == d) {
      lo[e] = 0;
      hi[e] = c.n[e] + 1;
    } else if (c.n[e] > 1) {
      lo[e] = -1;
      hi[e] = c.n[e] + 1;
    } else {
      lo[e] = 0;
      hi[e] = 1;
    }
  }
  std::vector<double>& F = c.F[d];
  std::fill(F.begin(), F.end(), 0.0);
  std::fill(c.spd[d].begin(), c.spd[d].end(), 0.0);
  long str = d == 0 ? 1 : (d == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
  auto one_face = [&](int i, int j, int k) {
    int ii[3] = {i, j, k};
    int f = ii[d];
    long t = idx(c, i, j, k);  // cell just above the face
    // polar faces: sqrt(-g) = 0 there, flux is zero
    if (p.metric == 1 && d == 1 &&
        ((f == 0 && p.bc[2] == 2) || (f == c.n[1] && p.bc[3] == 2)))
      return;
    double P8[8][NP], K8[8];
    const Geom* geo[8];
    for (int m = 0; m < 8; ++m) {
      long cm = t + (long)(m - 4) * str;
      geo[m] = &c.geo[cm];
      for (int q = 0; q < NP; ++q) P8[m][q] = c.P[(long)q * c.ntot + cm];
      K8[m] = c.K.empty() ? 0.0 : c.K[cm];
    }
    double x[3] = {xc(c, 0, i), xc(c, 1, j), xc(c, 2, k)};
    x[d] = xf(c, d, f);
    Geom G;
    geom_at(p, x[0], x[1], x[2], G);
    double* st[2][2] = {{&c.flat[d][t - str], &c.flat[d][c.ntot + t - str]},
                        {&c.flat[d][t], &c.flat[d][c.ntot + t]}};
    double Fq[NP], sp, fs = 0.0, gs[2];
    face_flux(p, d, P8, geo, G, c.K.empty() ? nullptr : K8, use_stored ? st : nullptr, Fq, &sp,
              p.integrator == 0 ? &fs : nullptr, gs);
    for (int q = 0; q < NP; ++q) F[(long)q * c.ntot + t] = Fq[q];
    c.spd[d][t] = sp;
    c.FS[d][t] = fs;
    if (!c.gsp[d].empty()) {
      c.gsp[d][t] = gs[0];
      c.gsp[d][c.ntot + t] = gs[1];
    }
  };
  // a face writes the flattener of the two cells beside it: the parallel
  // loop runs over an index other than d, so neighbours along d stay on one
  // thread
  const int nth = orc_threads();
  if (d != 2) {
#pragma omp parallel for num_threads(nth) schedule(dynamic, 1)
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) one_face(i, j, k);
  } else {
#pragma omp parallel for num_threads(nth) schedule(dynamic, 1)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int i = lo[0]; i < hi[0]; ++i) one_face(i, j, k);
  }
}

// Flux-CT (Toth 2000): for every pair (a,b) of active directions, the edge
// EMF is the average of the four face fluxes that touch the edge, and the
// induction fluxes are replaced by averages of the two adjacent edge EMFs.
void flux_ct(Ctx& c) {
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      if (c.n[a] == 1 || c.n[b] == 1) continue;
      int e = 3 - a - b;
      long sa = a == 0 ? 1 : (a == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
      long sb = b == 0 ? 1 : (b == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
      std::vector<double> emf(c.ntot, 0.0);
      int lo[3] = {0, 0, 0}, hi[3];
      for (int z = 0; z < 3; ++z) hi[z] = c.n[z];
      hi[a] = c.n[a] + 1;
      hi[b] = c.n[b] + 1;
      const double* Fa = &c.F[a][(long)(B1 + b) * c.ntot];
      const double* Fb = &c.F[b][(long)(B1 + a) * c.ntot];
#pragma omp parallel for num_threads(orc_threads())
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            long t = idx(c, i, j, k);
            int ii[3] = {i, j, k};
            bool pole = false;
            if (c.p.metric == 1 && (a == 1 || b == 1)) {
              if ((ii[1] == 0 && c.p.bc[2] == 2) || (ii[1] == c.n[1] && c.p.bc[3] == 2)) pole = true;
            }
            (void)e;
            emf[t] = pole ? 0.0 : 0.25 * (Fa[t] + Fa[t - sb] - Fb[t] - Fb[t - sa]);
          }
      double* Fa_w = &c.F[a][(long)(B1 + b) * c.ntot];
      double* Fb_w = &c.F[b][(long)(B1 + a) * c.ntot];
      // F_a[B_b] on a-faces: a in [0,n_a], b in [0,n_b)
#pragma omp parallel for num_threads(orc_threads())
      for (int k = 0; k < (a == 2 ? c.n[2] + 1 : c.n[2]); ++k)
        for (int j = 0; j < (a == 1 ? c.n[1] + 1 : c.n[1]); ++j)
          for (int i = 0; i < (a == 0 ? c.n[0] + 1 : c.n[0]); ++i) {
            long t = idx(c, i, j, k);
            Fa_w[t] = 0.5 * (emf[t] + emf[t + sb]);
          }
#pragma omp parallel for num_threads(orc_threads())
      for (int k = 0; k < (b == 2 ? c.n[2] + 1 : c.n[2]); ++k)
        for (int j = 0; j < (b == 1 ? c.n[1] + 1 : c.n[1]); ++j)
          for (int i = 0; i < (b == 0 ? c.n[0] + 1 : c.n[0]); ++i) {
            long t = idx(c, i, j, k);
            Fb_w[t] = -0.5 * (emf[t] + emf[t + sa]);
          }
    }
  for (int d = 0; d < 3; ++d) {
    if (c.n[d] == 1) continue;
    double* Fd = &c.F[d][(long)(B1 + d) * c.ntot];
    for (long t = 0; t < c.ntot; ++t) Fd[t] = 0.0;
  }
}

// ------------------------------------------------------- staggered field
// With emf = 1 the magnetic field is evolved on cell faces (Sec. 4, the list
// of quantities; Sec. 4.2 steps viii-x): Bf[d] holds sqrt(-g) B^d on the
// lower d-face of each cell, the EMFs sit on the cell edges, and the
// cell-centred B of a zone is the average of its two faces' sqrt(-g) B^d
// divided by the centre's sqrt(-g).  A direction with one zone has one face
// per cell, the cell itself.

inline long stride(const Ctx& c, int d) { return d == 0 ? 1 : (d == 1 ? c.N[0] : (long)c.N[0] * c.N[1]); }
inline bool periodic(const Ctx& c, int d) { return c.p.bc[2 * d] == 0 && c.p.bc[2 * d + 1] == 0; }
// position of a cell's lower d-face along d (the centre when n_d = 1)
inline double xface(const Ctx& c, int d, int i) { return c.n[d] > 1 ? xf(c, d, i) : xc(c, d, i); }

// Index ranges of the evolved faces of direction d: along d, faces 0..n_d
// (0..n_d-1 when d is periodic: face n_d is face 0's image); across, the
// active zones.
void face_range(const Ctx& c, int d, int lo[3], int hi[3]) {
  for (int e = 0; e < 3; ++e) {
    lo[e] = 0;
    hi[e] = c.n[e];
  }
  if (c.n[d] > 1 && !periodic(c, d)) hi[d] = c.n[d] + 1;
}

// Faces outside the evolved ranges: the periodic image where one exists,
// else the average of the two cells beside the face of sqrt(-g) B^d (the
// ghost cells hold the boundary conditions' B), or the one cell inside the
// array on its outermost layer.
void fill_face_ghosts(Ctx& c) {
  for (int d = 0; d < 3; ++d) {
    int lo[3], hi[3];
    face_range(c, d, lo, hi);
    const long sd = stride(c, d);
    for (int k = -c.ng[2]; k < c.n[2] + c.ng[2]; ++k)
      for (int j = -c.ng[1]; j < c.n[1] + c.ng[1]; ++j)
        for (int i = -c.ng[0]; i < c.n[0] + c.ng[0]; ++i) {
          int ii[3] = {i, j, k};
          bool inside = true;
          for (int e = 0; e < 3; ++e) inside = inside && ii[e] >= lo[e] && ii[e] < hi[e];
          if (inside) continue;
          const long t = idx(c, i, j, k);
          int w[3] = {i, j, k};
          bool image = true;
          for (int e = 0; e < 3; ++e) {
            if (w[e] >= lo[e] && w[e] < hi[e]) continue;
            if (periodic(c, e) && c.n[e] > 1) w[e] = ((w[e] % c.n[e]) + c.n[e]) % c.n[e];
            else image = false;
          }
          if (image) {
            c.Bf[d][t] = c.Bf[d][idx(c, w[0], w[1], w[2])];
            continue;
          }
          const double bt = c.geo[t].gdet * c.P[(long)(B1 + d) * c.ntot + t];
          if (c.n[d] == 1 || ii[d] == -c.ng[d]) {
            c.Bf[d][t] = bt;
          } else {
            const double bm = c.geo[t - sd].gdet * c.P[(long)(B1 + d) * c.ntot + t - sd];
            c.Bf[d][t] = 0.5 * (bm + bt);
          }
        }
  }
}

// sqrt(-g) B^d at the centre of cell t from its faces.
inline double centre_flux(const Ctx& c, int d, long t) {
  return c.n[d] > 1 ? 0.5 * (c.Bf[d][t] + c.Bf[d][t + stride(c, d)]) : c.Bf[d][t];
}

// Cell-centred B of the active zones from the faces.
void centre_B_from_faces(Ctx& c) {
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        long t = idx(c, i, j, k);
        for (int d = 0; d < 3; ++d) c.P[(long)(B1 + d) * c.ntot + t] = centre_flux(c, d, t) / c.geo[t].gdet;
      }
}

// Faces from the cell-centred B: sqrt(-g) B^d averaged over the two cells
// beside each evolved face (after the ghost fill), then the centres from the
// faces.
void faces_from_centres(Ctx& c) {
  fill_ghosts(c, c.P);
  for (int d = 0; d < 3; ++d) {
    const long sd = stride(c, d);
    for (int k = -c.ng[2]; k < c.n[2] + c.ng[2]; ++k)
      for (int j = -c.ng[1]; j < c.n[1] + c.ng[1]; ++j)
        for (int i = -c.ng[0]; i < c.n[0] + c.ng[0]; ++i) {
          const int ii[3] = {i, j, k};
          const long t = idx(c, i, j, k);
          const double bt = c.geo[t].gdet * c.P[(long)(B1 + d) * c.ntot + t];
          if (c.n[d] == 1 || ii[d] == -c.ng[d]) c.Bf[d][t] = bt;
          else c.Bf[d][t] = 0.5 * (c.geo[t - sd].gdet * c.P[(long)(B1 + d) * c.ntot + t - sd] + bt);
        }
  }
  fill_face_ghosts(c);
  centre_B_from_faces(c);
}

// 4-state upwind EMF (Sec. 4.2 steps viii-ix, after Del Zanna et al. 2007)
// for every pair a < b of directions of which one has more than one zone, on
// the edges (lower a-face, lower b-face) of the cells:
//   emf_ab = sqrt(-g) (B^b v^a - B^a v^b), the flux of sqrt(-g) B^b along a
//   and minus that of sqrt(-g) B^a along b.
// The field components come from the faces: B^b from the b-faces on either
// side of the edge along a, interpolated to the edge along a (MC-limited
// linear), and B^a likewise along b.  The velocities v^i = u^i/u^t of the
// four cells around the edge are extrapolated to it with MC-limited slopes.
// The signal speeds along a at the edge interpolate (average) the gas
// speeds v_max, v_min of the two a-faces beside it, and likewise along b.
// The four states are combined by the 2D HLL (or, with LAXF, by weights
// v_tot), with the dissipation of each direction's 1D HLL/LAXF flux
// (Eqs. hll, lax).  Edges on the polar axis carry no EMF.
void uct_emfs(Ctx& c, std::vector<double> emf[3]) {
  const orc_params& p = c.p;
  // v^i of every cell
  std::vector<double> V((size_t)3 * c.ntot, 0.0);
  for (long t = 0; t < c.ntot; ++t) {
    double ut[3] = {c.P[(long)U1 * c.ntot + t], c.P[(long)U2 * c.ntot + t], c.P[(long)U3 * c.ntot + t]};
    FourVel u;
    fourvel(c.geo[t], ut, u);
    for (int i = 0; i < 3; ++i) V[(long)i * c.ntot + t] = u.ucon[i + 1] / u.ucon[0];
  }
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      const int e = 3 - a - b;
      std::vector<double>& E = emf[e];
      E.assign((size_t)c.ntot, 0.0);
      if (c.n[a] == 1 && c.n[b] == 1) continue;
      const long sa = stride(c, a), sb = stride(c, b);
      const bool aa = c.n[a] > 1, ab = c.n[b] > 1;
      int hi[3];
      for (int z = 0; z < 3; ++z) hi[z] = c.n[z];
      if (aa) hi[a] = c.n[a] + 1;
      if (ab) hi[b] = c.n[b] + 1;
      // face primitive B^d = Bf / sqrt(-g) at the face position
      auto Bface = [&](int d, long t, int i, int j, int k) {
        double x[3] = {xc(c, 0, i), xc(c, 1, j), xc(c, 2, k)};
        int ii[3] = {i, j, k};
        x[d] = xface(c, d, ii[d]);
        Geom G;
        geom_at(p, x[0], x[1], x[2], G);
        return c.Bf[d][t] / G.gdet;
      };
      for (int k = 0; k < hi[2]; ++k)
        for (int j = 0; j < hi[1]; ++j)
          for (int i = 0; i < hi[0]; ++i) {
            const long t = idx(c, i, j, k);
            const int ii[3] = {i, j, k};
            if (p.metric == 1 && (a == 1 || b == 1) &&
                ((j == 0 && p.bc[2] == 2) || (j == c.n[1] && p.bc[3] == 2)))
              continue;  // polar axis
            double x[3] = {xc(c, 0, i), xc(c, 1, j), xc(c, 2, k)};
            x[a] = xface(c, a, ii[a]);
            x[b] = xface(c, b, ii[b]);
            Geom Ge;
            geom_at(p, x[0], x[1], x[2], Ge);
            // B^b along a (sides - and + of the edge), B^a along b
            // face value B^d of the cell offset by o along direction m
            auto Bat = [&](int d, int m, int o) {
              int q[3] = {i, j, k};
              q[m] += o;
              return Bface(d, t + o * stride(c, m), q[0], q[1], q[2]);
            };
            double Bb[2], Ba[2];
            {
              const double b0 = Bat(b, a, 0);
              if (aa) {
                const double bmm = Bat(b, a, -2), bm = Bat(b, a, -1), bp = Bat(b, a, 1);
                Bb[0] = bm + 0.5 * mc_slope(bmm, bm, b0);
                Bb[1] = b0 - 0.5 * mc_slope(bm, b0, bp);
              } else {
                Bb[0] = Bb[1] = b0;
              }
            }
            {
              const double b0 = Bat(a, b, 0);
              if (ab) {
                const double bmm = Bat(a, b, -2), bm = Bat(a, b, -1), bp = Bat(a, b, 1);
                Ba[0] = bm + 0.5 * mc_slope(bmm, bm, b0);
                Ba[1] = b0 - 0.5 * mc_slope(bm, b0, bp);
              } else {
                Ba[0] = Ba[1] = b0;
              }
            }
            // the four corner states: side sa_ (0: -, 1: +) along a, sb_ along b
            double es[2][2];
            for (int s1 = 0; s1 < 2; ++s1)
              for (int s2 = 0; s2 < 2; ++s2) {
                const long tc = t - (s1 == 0 && aa ? sa : 0) - (s2 == 0 && ab ? sb : 0);
                double v[2];
                const int comp[2] = {a, b};
                for (int m = 0; m < 2; ++m) {
                  const double* Vm = &V[(long)comp[m] * c.ntot];
                  double val = Vm[tc];
                  if (aa) val += (s1 == 0 ? 0.5 : -0.5) * mc_slope(Vm[tc - sa], Vm[tc], Vm[tc + sa]);
                  if (ab) val += (s2 == 0 ? 0.5 : -0.5) * mc_slope(Vm[tc - sb], Vm[tc], Vm[tc + sb]);
                  v[m] = val;
                }
                es[s1][s2] = Ge.gdet * (Bb[s1] * v[0] - Ba[s2] * v[1]);
              }
            // signal speeds at the edge and the weights of each side
            double wa[2] = {0.0, 0.0}, wb[2] = {0.0, 0.0};
            if (aa) {
              const long f0 = ab ? t - sb : t;
              const double vmax = 0.5 * (c.gsp[a][f0] + c.gsp[a][t]);
              const double vmin = 0.5 * (c.gsp[a][c.ntot + f0] + c.gsp[a][c.ntot + t]);
              if (p.flux == 0) wa[0] = wa[1] = std::max(vmax, vmin);
              else {
                wa[0] = vmax;
                wa[1] = vmin;
              }
            }
            if (ab) {
              const long f0 = aa ? t - sa : t;
              const double vmax = 0.5 * (c.gsp[b][f0] + c.gsp[b][t]);
              const double vmin = 0.5 * (c.gsp[b][c.ntot + f0] + c.gsp[b][c.ntot + t]);
              if (p.flux == 0) wb[0] = wb[1] = std::max(vmax, vmin);
              else {
                wb[0] = vmax;
                wb[1] = vmin;
              }
            }
            double Wa = wa[0] + wa[1], Wb = wb[0] + wb[1];
            double da = 0.0, db = 0.0;
            if (Wa > 0.0) da = wa[0] * wa[1] / Wa;
            else wa[0] = wa[1] = Wa = 1.0;
            if (Wb > 0.0) db = wb[0] * wb[1] / Wb;
            else wb[0] = wb[1] = Wb = 1.0;
            double sum = 0.0;
            for (int s1 = 0; s1 < 2; ++s1)
              for (int s2 = 0; s2 < 2; ++s2) sum += wa[s1] * wb[s2] * es[s1][s2];
            E[t] = sum / (Wa * Wb) - da * Ge.gdet * (Bb[1] - Bb[0]) + db * Ge.gdet * (Ba[1] - Ba[0]);
          }
    }
}

// Right-hand side of the evolved face fields from the edge EMFs:
// d(sqrt(-g) B^d)/dt = - sum_{a != d} d_a emf_{a d}, emf_{a d} = -emf_{d a}.
void face_rhs(const Ctx& c, const std::vector<double> emf[3], int d, long t, double* rhs) {
  double r = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (a == d || c.n[a] == 1) continue;
    const int e = 3 - a - d;
    const double sgn = a < d ? 1.0 : -1.0;  // emf[e] holds emf_{min(a,d) max(a,d)}
    r -= sgn * (emf[e][t + stride(c, a)] - emf[e][t]) / c.p.dx[a];
  }
  *rhs = r;
}

// Floors (Sec. 2 and Sec. 4.11; values from the configuration): Lorentz
// factor caps, density and internal-energy floors, magnetisation caps and the
// positivity of Ebar.
void apply_floors(const orc_params& p, const Geom& G, double* P) {
  double ut[3] = {P[U1], P[U2], P[U3]};
  FourVel u;
  fourvel(G, ut, u);
  if (u.gamma > p.gamma_gas_max) {
    double f = std::sqrt((p.gamma_gas_max * p.gamma_gas_max - 1.0) / (u.gamma * u.gamma - 1.0));
    for (int i = 0; i < 3; ++i) P[U1 + i] *= f;
  }
  double ur[3] = {P[UR1], P[UR2], P[UR3]};
  FourVel v;
  fourvel(G, ur, v);
  if (v.gamma > p.gamma_rad_max) {
    double f = std::sqrt((p.gamma_rad_max * p.gamma_rad_max - 1.0) / (v.gamma * v.gamma - 1.0));
    for (int i = 0; i < 3; ++i) P[UR1 + i] *= f;
  }
  double ut2[3] = {P[U1], P[U2], P[U3]};
  fourvel(G, ut2, u);
  double B[3] = {P[B1], P[B2], P[B3]}, bcon[4], bcov[4], bsq;
  bfield(G, u, B, bcon, bcov, &bsq);
  double rfl = std::max(p.floor_rho0 * std::pow(G.r, p.floor_rho_pow), bsq / p.bsq_rho_max);
  double ufl = std::max(p.floor_u0 * std::pow(G.r, p.floor_u_pow), bsq / p.bsq_u_max);
  P[RHO] = std::max(P[RHO], rfl);
  P[UU] = std::max(P[UU], ufl);
  P[RHO] = std::max(P[RHO], P[UU] / p.u_rho_max);
  if (!(P[ER] > 0.0)) P[ER] = 1e-150;
}

double cfl_from_speeds(const Ctx& c) {
  double best = HUGE_VAL;
#pragma omp parallel for num_threads(orc_threads()) reduction(min : best)
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        long t = idx(c, i, j, k);
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (c.n[d] == 1) continue;
          long st = d == 0 ? 1 : (d == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
          double v = std::max(c.spd[d][t], c.spd[d][t + st]);
          s += v / c.p.dx[d];
        }
        if (s > 0.0) best = std::min(best, 1.0 / s);
      }
  return c.p.courant * best;
}

double cfl_dt(Ctx& c) {
  fill_ghosts(c, c.P);
  for (int d = 0; d < 3; ++d)
    if (c.n[d] > 1) compute_fluxes(c, d, false);
  return cfl_from_speeds(c);
}

// Stage k of an IMEX scheme of Sec. 4.1 in the paper's bracket form: the
// explicit part U* = an U^n + ap U(P) + d dt F(P) + dt sum_j c_j M^j, with P
// the primitives the previous stage left and F the explicit right-hand side
// (flux divergence and geometric source) at P, then the implicit stage
// U = U* + g dt M(U); the final combination has g = 0 (the conserved state is
// only inverted).  M^j is the implicit source of stage j: +G on the gas
// energy-momentum rows, -G on the radiation rows.
struct Pass {
  double an, ap, d, c[4], g;
};

int n_passes(int integrator) {
  static const int n[4] = {3, 3, 4, 5};
  return n[integrator];
}

Pass imex_pass(int integrator, int k) {
  Pass s = {0.0, 0.0, 0.0, {0.0, 0.0, 0.0, 0.0}, 0.0};
  if (integrator == 1) {
    // IMEX2, gamma = 1 - 1/sqrt(2)
    const double ga = 1.0 - 1.0 / std::sqrt(2.0);
    if (k == 0) {  // U^0 = [U^n] + gamma dt M^0
      s.an = 1.0;
      s.g = ga;
    } else if (k == 1) {  // U^1 = [(3gamma-1)/gamma U^n + (1-2gamma)/gamma U^0 + dt F^0] + gamma dt M^1
      s.an = (3.0 * ga - 1.0) / ga;
      s.ap = (1.0 - 2.0 * ga) / ga;
      s.d = 1.0;
      s.g = ga;
    } else {  // U^{n+1} = [U^n/2 + U^1/2 + dt/2 F^1 + gamma dt M^0 + (1-gamma)/2 dt M^1]
      s.an = 0.5;
      s.ap = 0.5;
      s.d = 0.5;
      s.c[0] = ga;
      s.c[1] = 0.5 * (1.0 - ga);
    }
  } else if (integrator == 2) {
    // IMEX2B
    if (k == 0) {  // U^0 = [U^n] + dt/4 M^0
      s.an = 1.0;
      s.g = 0.25;
    } else if (k == 1) {  // U^1 = [U^n + dt/2 F^0] + dt/4 M^1
      s.an = 1.0;
      s.d = 0.5;
      s.g = 0.25;
    } else if (k == 2) {  // U^2 = [U^1 + dt/2 F^1 + dt/3 M^0 + dt/12 M^1] + dt/3 M^2
      s.ap = 1.0;
      s.d = 0.5;
      s.c[0] = 1.0 / 3.0;
      s.c[1] = 1.0 / 12.0;
      s.g = 1.0 / 3.0;
    } else {  // U^{n+1} = [U^n/3 + 2U^2/3 + dt/3 F^2 + dt/9 (M^0 + M^1 + M^2)]
      s.an = 1.0 / 3.0;
      s.ap = 2.0 / 3.0;
      s.d = 1.0 / 3.0;
      s.c[0] = s.c[1] = s.c[2] = 1.0 / 9.0;
    }
  } else if (integrator == 3) {
    // IMEX3 with the printed alpha, beta, eta
    const double al = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
    if (k == 0) {  // U^0 = [U^n] + alpha dt M^0
      s.an = 1.0;
      s.g = al;
    } else if (k == 1) {  // U^1 = [2U^n - U^0] + alpha dt M^1, with the bracket taken as
                          // [U^n - alpha dt M^0]: equal by the first stage, but free of
                          // the floors' additions to U^0, which 2U^n - U^0 would subtract
      s.an = 1.0;
      s.c[0] = -al;
      s.g = al;
    } else if (k == 2) {  // U^2 = [U^n + dt F^1 + (1-alpha) dt M^1] + alpha dt M^2
      s.an = 1.0;
      s.d = 1.0;
      s.c[1] = 1.0 - al;
      s.g = al;
    } else if (k == 3) {  // U^3 = [3U^n/4 + U^2/4 + dt/4 F^2 + beta dt M^0
                          //        + (-1+alpha+4eta)/4 dt M^1 + (2-5alpha-4(beta+eta))/4 dt M^2] + alpha dt M^3
      s.an = 0.75;
      s.ap = 0.25;
      s.d = 0.25;
      s.c[0] = be;
      s.c[1] = (-1.0 + al + 4.0 * et) / 4.0;
      s.c[2] = (2.0 - 5.0 * al - 4.0 * (be + et)) / 4.0;
      s.g = al;
    } else {  // U^{n+1} = [U^n/3 + 2U^3/3 + 2dt/3 F^3 - 2beta/3 dt M^0 + (1-4eta)/6 dt M^1
              //            + (-1+4alpha+4(beta+eta))/6 dt M^2 + 4(1-alpha)/6 dt M^3]
      s.an = 1.0 / 3.0;
      s.ap = 2.0 / 3.0;
      s.d = 2.0 / 3.0;
      s.c[0] = -2.0 * be / 3.0;
      s.c[1] = (1.0 - 4.0 * et) / 6.0;
      s.c[2] = (-1.0 + 4.0 * al + 4.0 * (be + et)) / 6.0;
      s.c[3] = 4.0 * (1.0 - al) / 6.0;
    }
  }
  return s;
}

// One sub-step s (Sec. 4.1-4.2): an RK3 stage, or stage s of an IMEX scheme.
void substep(Ctx& c, int s, double dt) {
  static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double Bc[3] = {1.0, 0.25, 2.0 / 3.0};
  const bool imex = c.p.integrator != 0;
  const Pass ps = imex_pass(c.p.integrator, s);
  // an IMEX stage without an explicit right-hand side needs no fluxes
  const bool rhs = !imex || ps.d != 0.0;
  const bool uct = c.p.emf == 1;
  std::vector<double> emf[3];
  if (rhs) {
    fill_ghosts(c, c.P);
    if (uct) fill_face_ghosts(c);
    for (int d = 0; d < 3; ++d)
      if (c.n[d] > 1) compute_fluxes(c, d, c.p.recon == 0);
    if (uct) uct_emfs(c, emf);
    else flux_ct(c);
  }
  if (uct) {
    // the staggered field's stage (Sec. 4.2 step x): the same combination as
    // the cell-centred conserved quantities, with the EMFs' curl for X
    for (int d = 0; d < 3; ++d) {
      if (s == 0) c.Bfn[d] = c.Bf[d];
      int lo[3], hi[3];
      face_range(c, d, lo, hi);
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            const long t = idx(c, i, j, k);
            double r = 0.0;
            if (rhs) face_rhs(c, emf, d, t, &r);
            const double bn = c.Bfn[d][t], bs = c.Bf[d][t];
            c.Bf[d][t] = !imex ? A[s] * bn + Bc[s] * (bs + dt * r) : ps.an * bn + ps.ap * bs + ps.d * dt * r;
          }
    }
    fill_face_ghosts(c);
  }
  std::vector<double> Pnew((size_t)NP * c.ntot);
  std::memcpy(Pnew.data(), c.P.data(), sizeof(double) * NP * c.ntot);
  std::vector<unsigned char> failed((size_t)c.n[0] * c.n[1] * c.n[2], 0);
  long long n_pmhd = 0, n_urad = 0, n_back = 0, n_iter = 0, n_solve = 0, n_ent = 0, n_cold = 0;
#pragma omp parallel for num_threads(orc_threads()) schedule(dynamic, 1) \
    reduction(+ : n_pmhd, n_urad, n_back, n_iter, n_solve, n_ent, n_cold)
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        long t = idx(c, i, j, k);
        const Geom& G = c.geo[t];
        double Ps[NP], Us[NP], SM[NP], X[NP], Ust[NP];
        for (int q = 0; q < NP; ++q) Ps[q] = c.P[(long)q * c.ntot + t];
        const double(*Gam)[4][4] = reinterpret_cast<const double(*)[4][4]>(&c.gam[(size_t)t * 64]);
        prim_to_cons(c.p, G, Gam, Ps, Us, SM);
        if (s == 0)
          for (int q = 0; q < NP; ++q) c.Un[(long)q * c.ntot + t] = Us[q];
        for (int q = 0; q < NP; ++q) {
          X[q] = 0.0;
          if (rhs) {
            double div = 0.0;
            for (int d = 0; d < 3; ++d) {
              if (c.n[d] == 1) continue;
              long st = d == 0 ? 1 : (d == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
              div += (c.F[d][(long)q * c.ntot + t + st] - c.F[d][(long)q * c.ntot + t]) / c.p.dx[d];
            }
            X[q] = -div + SM[q];
          }
          if (uct && q >= B1 && q <= B3) {
            Ust[q] = centre_flux(c, q - B1, t);  // the field from the evolved faces
          } else if (!imex) {
            Ust[q] = A[s] * c.Un[(long)q * c.ntot + t] + Bc[s] * (Us[q] + dt * X[q]);
          } else {
            double v = ps.an * c.Un[(long)q * c.ntot + t] + ps.ap * Us[q] + ps.d * dt * X[q];
            // earlier stages' implicit sources: +M on the gas rows, -M on the radiation rows
            int row = -1;
            double sg = 0.0;
            if (q >= UU && q <= U3) {
              row = q - UU;
              sg = 1.0;
            } else if (q >= ER && q <= UR3) {
              row = q - ER;
              sg = -1.0;
            }
            if (row >= 0)
              for (int j = 0; j < s; ++j) v += dt * ps.c[j] * sg * c.M[j][(long)row * c.ntot + t];
            Ust[q] = v;
          }
        }
        // RK3: the explicit entropy S* = a_s S^n + b_s (S(P_s) + dt X_S), the
        // conserved entropy sqrt(-g) S u^t = U_rho s_gas (Sec. 2, Eq. S), for the
        // entropy equation of the implicit solve (Sec. 4.7, 4.11)
        double Sst = 0.0;
        if (!imex) {
          const double Su = Us[RHO] * entropy_per_baryon(c.p, Ps[RHO], Ps[UU]);
          if (s == 0) c.Sn[t] = Su;
          double divS = 0.0;
          for (int d = 0; d < 3; ++d) {
            if (c.n[d] == 1) continue;
            long st = d == 0 ? 1 : (d == 1 ? c.N[0] : (long)c.N[0] * c.N[1]);
            divS += (c.FS[d][t + st] - c.FS[d][t]) / c.p.dx[d];
          }
          Sst = A[s] * c.Sn[t] + Bc[s] * (Su - dt * divS);
        }
        double Pn[NP];
        orc_implicit_info info;
        const double h = imex ? ps.g * dt : Bc[s] * dt;
        implicit_zone(cell_params(c, t), G, Ust, imex ? nullptr : &Sst, Ps, h, Pn, &info,
                      radiation_subdominant(G, Ust, Ps));
        if (imex && ps.g > 0.0) {
          // M^s = (U(P) - U*) / (g dt) on the gas rows, P the implicit stage's
          // solution (the source as the change the implicit stage made)
          double Uz[NP], SMz[NP];
          prim_to_cons(c.p, G, Gam, Pn, Uz, SMz);
          for (int r = 0; r < 4; ++r) c.M[s][(long)r * c.ntot + t] = (Uz[UU + r] - Ust[UU + r]) / h;
        }
        long a = aidx(c, i, j, k);
        c.status[a] = std::max(c.status[a], (unsigned char)info.method);
        c.iters[a] += info.iters_pmhd + info.iters_urad;
        n_iter += info.iters_pmhd + info.iters_urad;
        n_solve += 1;
        n_ent += info.entropy;
        n_cold += info.cold;
        if (info.method == ORC_OK_PMHD) n_pmhd++;
        else if (info.method == ORC_OK_URAD) n_urad++;
        else n_back++;
        failed[a] = info.method == ORC_BACKUP ? 1 : (info.cold ? 2 : 0);
        apply_floors(c.p, G, Pn);
        for (int q = 0; q < NP; ++q) Pnew[(long)q * c.ntot + t] = Pn[q];
      }
  c.counts[0] += n_pmhd;
  c.counts[1] += n_urad;
  c.counts[2] += n_back;
  c.counts[3] += n_iter;
  c.counts[4] += n_solve;
  c.counts[5] += n_ent;
  c.counts[6] += n_cold;
  // Back-up (Sec. 4.11): replace failed zones by the average of their good
  // active face neighbours (all active neighbours if none is good); B keeps
  // its constrained-transport value.  A zone solved by the cold-MHD equations
  // has only its u_g replaced by that average, and counts as not good for its
  // neighbours.  All averages are taken from the solutions before any is
  // replaced.  Every solution was floored above, and the floors are applied
  // once more after averaging (they are idempotent).
  std::vector<double> Pavg = Pnew;
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        if (!failed[aidx(c, i, j, k)]) continue;
        long t = idx(c, i, j, k);
        double sum_good[NP] = {0}, sum_all[NP] = {0};
        int ngood = 0, nall = 0;
        for (int d = 0; d < 3; ++d) {
          if (c.n[d] == 1) continue;
          for (int side = -1; side <= 1; side += 2) {
            int nb[3] = {i, j, k};
            nb[d] += side;
            if (nb[d] < 0 || nb[d] >= c.n[d]) continue;
            long tn = idx(c, nb[0], nb[1], nb[2]);
            bool good = !failed[aidx(c, nb[0], nb[1], nb[2])];
            for (int q = 0; q < NP; ++q) {
              double v = Pnew[(long)q * c.ntot + tn];
              sum_all[q] += v;
              if (good) sum_good[q] += v;
            }
            nall++;
            if (good) ngood++;
          }
        }
        if (nall == 0) continue;
        const bool cold = failed[aidx(c, i, j, k)] == 2;
        for (int q = 0; q < NP; ++q) {
          if (q >= B1 && q <= B3) continue;
          if (cold && q != UU) continue;
          Pavg[(long)q * c.ntot + t] = ngood > 0 ? sum_good[q] / ngood : sum_all[q] / nall;
        }
      }
#pragma omp parallel for num_threads(orc_threads())
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        long t = idx(c, i, j, k);
        double Pz[NP];
        for (int q = 0; q < NP; ++q) Pz[q] = Pavg[(long)q * c.ntot + t];
        apply_floors(c.p, c.geo[t], Pz);
        for (int q = 0; q < NP; ++q) c.P[(long)q * c.ntot + t] = Pz[q];
      }
}

}  // namespace
}  // namespace orc

using namespace orc;

extern "C" {

void* orc_create(const orc_params* p) {
  Ctx* c = new Ctx();
  c->p = *p;
  if (c->p.newton_max > 60) c->p.newton_max = 60;
  c->ntot = 1;
  for (int d = 0; d < 3; ++d) {
    c->n[d] = p->n[d];
    c->ng[d] = p->n[d] > 1 ? NG : 0;
    c->N[d] = c->n[d] + 2 * c->ng[d];
    c->ntot *= c->N[d];
  }
  c->P.assign((size_t)NP * c->ntot, 0.0);
  if (p->opacity == 2) c->K.assign((size_t)c->ntot, 0.0);
  c->Un.assign((size_t)NP * c->ntot, 0.0);
  c->Sn.assign((size_t)c->ntot, 0.0);
  for (int d = 0; d < 3; ++d) {
    c->F[d].assign((size_t)NP * c->ntot, 0.0);
    c->spd[d].assign((size_t)c->ntot, 0.0);
    c->FS[d].assign((size_t)c->ntot, 0.0);
    c->flat[d].assign((size_t)2 * c->ntot, 0.0);
  }
  if (c->p.integrator < 0 || c->p.integrator > 3) c->p.integrator = 0;
  if (c->p.emf == 1)
    for (int d = 0; d < 3; ++d) {
      c->Bf[d].assign((size_t)c->ntot, 0.0);
      c->Bfn[d].assign((size_t)c->ntot, 0.0);
      c->gsp[d].assign((size_t)2 * c->ntot, 0.0);
    }
  else
    c->p.emf = 0;
  if (c->p.integrator != 0)
    for (int j = 0; j < 4; ++j) c->M[j].assign((size_t)4 * c->ntot, 0.0);
  c->geo.resize(c->ntot);
  c->gam.assign((size_t)c->ntot * 64, 0.0);
#pragma omp parallel for num_threads(orc_threads()) schedule(dynamic, 1)
  for (int k = -c->ng[2]; k < c->n[2] + c->ng[2]; ++k)
    for (int j = -c->ng[1]; j < c->n[1] + c->ng[1]; ++j)
      for (int i = -c->ng[0]; i < c->n[0] + c->ng[0]; ++i) {
        long t = idx(*c, i, j, k);
        double x1 = xc(*c, 0, i), x2 = xc(*c, 1, j), x3 = xc(*c, 2, k);
        geom_at(c->p, x1, x2, x3, c->geo[t]);
        double G4[4][4][4];
        connection_at(c->p, x1, x2, x3, G4);
        std::memcpy(&c->gam[(size_t)t * 64], G4, sizeof(G4));
      }
  long na = (long)c->n[0] * c->n[1] * c->n[2];
  c->status.assign(na, 0);
  c->iters.assign(na, 0);
  for (int i = 0; i < 7; ++i) c->counts[i] = 0;
  return c;
}

void orc_destroy(void* ctx) { delete static_cast<Ctx*>(ctx); }

void orc_set_prims(void* ctx, const double* P) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  long na = (long)c.n[0] * c.n[1] * c.n[2];
  for (int q = 0; q < NP; ++q)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i)
          c.P[(long)q * c.ntot + idx(c, i, j, k)] = P[(long)q * na + aidx(c, i, j, k)];
  if (c.p.emf == 1) faces_from_centres(c);
}

void orc_set_prims_with_ghosts(void* ctx, const double* P) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  for (long m = 0; m < (long)NP * c.ntot; ++m) c.P[m] = P[m];
  if (c.p.emf == 1) faces_from_centres(c);
}

// Active face layout of direction d: [n3'][n2'][n1'], n_d' = n_d + 1 if
// n_d > 1 (else 1), n_e' = n_e across.
static void face_dims(const Ctx& c, int d, int m[3]) {
  for (int e = 0; e < 3; ++e) m[e] = c.n[e];
  if (c.n[d] > 1) m[d] = c.n[d] + 1;
}

void orc_set_face_fields(void* ctx, const double* Bf) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  if (c.p.emf != 1) return;
  fill_ghosts(c, c.P);
  long off = 0;
  for (int d = 0; d < 3; ++d) {
    int m[3];
    face_dims(c, d, m);
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i) c.Bf[d][idx(c, i, j, k)] = Bf[off + ((long)k * m[1] + j) * m[0] + i];
    off += (long)m[0] * m[1] * m[2];
  }
  fill_face_ghosts(c);
  centre_B_from_faces(c);
}

void orc_get_face_fields(void* ctx, double* Bf) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  if (c.p.emf != 1) return;
  long off = 0;
  for (int d = 0; d < 3; ++d) {
    int m[3];
    face_dims(c, d, m);
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i) Bf[off + ((long)k * m[1] + j) * m[0] + i] = c.Bf[d][idx(c, i, j, k)];
    off += (long)m[0] * m[1] * m[2];
  }
}

void orc_set_opacity_field(void* ctx, const double* K) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  if (c.K.empty()) return;
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) c.K[idx(c, i, j, k)] = K[aidx(c, i, j, k)];
}

void orc_get_prims(void* ctx, double* P) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  long na = (long)c.n[0] * c.n[1] * c.n[2];
  for (int q = 0; q < NP; ++q)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i)
          P[(long)q * na + aidx(c, i, j, k)] = c.P[(long)q * c.ntot + idx(c, i, j, k)];
}

void orc_get_prims_with_ghosts(void* ctx, double* P, int fill) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  if (fill) fill_ghosts(c, c.P);
  std::memcpy(P, c.P.data(), sizeof(double) * NP * c.ntot);
}

double orc_cfl_dt(void* ctx) { return cfl_dt(*static_cast<Ctx*>(ctx)); }

double orc_step(void* ctx, double dt) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  if (!(dt > 0.0)) dt = cfl_dt(c);
  for (int d = 0; d < 3; ++d) std::fill(c.flat[d].begin(), c.flat[d].end(), 0.0);
  std::fill(c.iters.begin(), c.iters.end(), 0);
  std::fill(c.status.begin(), c.status.end(), 0);
  for (int i = 0; i < 7; ++i) c.counts[i] = 0;
  for (int s = 0; s < n_passes(c.p.integrator); ++s) substep(c, s, dt);
  return dt;
}

void orc_get_status(void* ctx, unsigned char* st) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  std::memcpy(st, c.status.data(), c.status.size());
}

void orc_get_iters(void* ctx, int* it) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  std::memcpy(it, c.iters.data(), sizeof(int) * c.iters.size());
}

void orc_get_counts(void* ctx, long long* out) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  for (int i = 0; i < 7; ++i) out[i] = c.counts[i];
}

void orc_compute_fluxes(void* ctx, int dir, double* Fout) {
  Ctx& c = *static_cast<Ctx*>(ctx);
  fill_ghosts(c, c.P);
  for (int d = 0; d < 3; ++d) std::fill(c.flat[d].begin(), c.flat[d].end(), 0.0);
  for (int d = 0; d < 3; ++d)
    if (c.n[d] > 1) compute_fluxes(c, d, false);
  flux_ct(c);
  int d = dir - 1;
  int m[3] = {c.n[0], c.n[1], c.n[2]};
  m[d] += 1;
  long nf = (long)m[0] * m[1] * m[2];
  for (int q = 0; q < NP; ++q)
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i)
          Fout[(long)q * nf + ((long)k * m[1] + j) * m[0] + i] = c.F[d][(long)q * c.ntot + idx(c, i, j, k)];
}

void orc_metric(const orc_params* p, const double* x, double* gcov, double* gcon, double* gdet,
                double* alpha) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  std::memcpy(gcov, G.gcov, sizeof(G.gcov));
  std::memcpy(gcon, G.gcon, sizeof(G.gcon));
  *gdet = G.gdet;
  *alpha = G.alpha;
}

void orc_connection(const orc_params* p, const double* x, double* gam) {
  double G4[4][4][4];
  connection_at(*p, x[1], x[2], x[3], G4);
  std::memcpy(gam, G4, sizeof(G4));
}

void orc_prim_to_cons(const orc_params* p, const double* x, const double* P, double* U,
                      double* SM) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  double G4[4][4][4];
  connection_at(*p, x[1], x[2], x[3], G4);
  prim_to_cons(*p, G, G4, P, U, SM);
}

void orc_flux(const orc_params* p, const double* x, int d, const double* P, double* F,
              double* speeds4) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  double U[NP];
  face_state(*p, G, d, P, U, F, speeds4);
}

void orc_stress(const orc_params* p, const double* x, const double* P, double* T16, double* R16) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  double T[4][4], R[4][4], bcon[4], bcov[4], bsq;
  FourVel u, ur;
  gas_stress(*p, G, P, T, u, bcon, bcov, &bsq);
  rad_stress(G, P, R, ur);
  std::memcpy(T16, T, sizeof(T));
  std::memcpy(R16, R, sizeof(R));
}

void orc_four_force(const orc_params* p, const double* x, const double* P, double* G4) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  double R[4][4];
  FourVel ur, u;
  rad_stress(G, P, R, ur);
  double ut[3] = {P[U1], P[U2], P[U3]};
  fourvel(G, ut, u);
  four_force(*p, G, P[RHO], P[UU], u, R, G4);
}

int orc_rad_invert(const orc_params* p, const double* x, const double* Rt, int limiter,
                   double* Prad) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  return rad_invert(*p, G, Rt, limiter, Prad);
}

int orc_gas_invert(const orc_params* p, const double* x, const double* U, const double* Pg,
                   double tol, double* Pout) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  return gas_invert(*p, G, U, Pg, tol, Pout);
}

int orc_radiation_subdominant(const orc_params* p, const double* x, const double* Ustar, const double* Ps) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  return radiation_subdominant(G, Ustar, Ps) ? 1 : 0;
}

int orc_cold_allowed(const orc_params* p, const double* x, const double* Ustar, const double* Ps) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  return cold_allowed(G, Ustar, Ps) ? 1 : 0;
}

void orc_implicit_zone(const orc_params* p, const double* x, const double* Ustar, const double* Sstar,
                       const double* Ps, double h, double* Pout, orc_implicit_info* info) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  implicit_zone(*p, G, Ustar, Sstar, Ps, h, Pout, info, radiation_subdominant(G, Ustar, Ps));
}

void orc_method_zone(const orc_params* p, const double* x, const double* Ustar, const double* Sstar,
                     const double* Ps, double h, int method, double* Pout, double* eT, int* iters) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  method_zone(*p, G, Ustar, Sstar, Ps, h, method, Pout, eT, iters);
}

void orc_pmhd_residual(const orc_params* p, const double* x, const double* Ustar, double h,
                       const double* xg, double* E4, double* eT, double* eI) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  pmhd_residual_public(*p, G, Ustar, h, xg, E4, eT, eI);
}

void orc_face_flux_stencil(const orc_params* p, int d, const double* S, const double* xc8,
                           const double* xfc, double* F, double* speed) {
  Geom G8[8];
  const Geom* geo[8];
  double P8[8][NP];
  for (int m = 0; m < 8; ++m) {
    geom_at(*p, xc8[3 * m], xc8[3 * m + 1], xc8[3 * m + 2], G8[m]);
    geo[m] = &G8[m];
    for (int q = 0; q < NP; ++q) P8[m][q] = S[NP * m + q];
  }
  Geom Gf;
  geom_at(*p, xfc[0], xfc[1], xfc[2], Gf);
  face_flux(*p, d - 1, P8, geo, Gf, nullptr, nullptr, F, speed);
}

void orc_apply_floors(const orc_params* p, const double* x, double* P) {
  Geom G;
  geom_at(*p, x[1], x[2], x[3], G);
  apply_floors(*p, G, P);
}

void orc_ppm_cell(const double* s5, double chi, double* aL, double* aR) { ppm_cell(s5, chi, aL, aR); }

double orc_mc_slope(double qm, double q0, double qp) { return mc_slope(qm, q0, qp); }

double orc_levermore_xi(double f) {
  double f2 = f * f;
  return (3.0 + 4.0 * f2) / (5.0 + 2.0 * std::sqrt(4.0 - 3.0 * f2));
}

}  // extern "C"
