// HARMRAD oracle internals -- TEST INFRASTRUCTURE ONLY (see oracle.h).
#ifndef HARMRAD_ORACLE_INTERNAL_H
#define HARMRAD_ORACLE_INTERNAL_H
#include "oracle.h"

namespace orc {

enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, ER, UR1, UR2, UR3, NP = 12 };
enum { LIM_BASIC = 0, LIM_TYPE2 = 2 };
extern const double EPSM;

struct Geom {
  double gcov[4][4], gcon[4][4];
  double gdet, alpha, r;
  double x[4];
};

struct FourVel {
  double ucon[4], ucov[4], gamma;
};

void geom_at(const orc_params& p, double x1, double x2, double x3, Geom& G);
void connection_at(const orc_params& p, double x1, double x2, double x3, double Gam[4][4][4]);
void lower(const Geom& G, const double vcon[4], double vcov[4]);
void fourvel(const Geom& G, const double ut[3], FourVel& u);
void bfield(const Geom& G, const FourVel& u, const double B[3], double bcon[4], double bcov[4],
            double* bsq);
void gas_stress(const orc_params& p, const Geom& G, const double* P, double T[4][4], FourVel& u,
                double bcon[4], double bcov[4], double* bsq);
void rad_stress(const Geom& G, const double* P, double R[4][4], FourVel& ur);
void opacity(const orc_params& p, double rho, double ug, double* kabs, double* ksca);
void four_force(const orc_params& p, const Geom& G, double rho, double ug, const FourVel& u,
                const double R[4][4], double Gcov[4]);
void prim_to_cons(const orc_params& p, const Geom& G, const double Gam[4][4][4], const double* P,
                  double* U, double* SM);
void char_speeds(const Geom& G, const double ucon[4], double c2, int d, double* vmin,
                 double* vmax);
void face_state(const orc_params& p, const Geom& G, int d, const double* P, double* U, double* F,
                double sp[4]);
int rad_invert(const orc_params& p, const Geom& G, const double Rt[4], int limiter, double out[4]);
double entropy_per_baryon(const orc_params& p, double rho, double ug);
int gas_invert(const orc_params& p, const Geom& G, const double* U, const double* Pg, double tol,
               double* out);

// Implicit four-force solve of one zone (Sec. 4.7-4.11).
bool radiation_subdominant(const Geom& G, const double* Ustar, const double* Ps);
bool cold_allowed(const Geom& G, const double* Ustar, const double* Ps);
void implicit_zone(const orc_params& p, const Geom& G, const double* Ustar, const double* Sstar,
                   const double* Ps,
                   double h, double* Pout, orc_implicit_info* info, bool subdominant);
void method_zone(const orc_params& p, const Geom& G, const double* Ustar, const double* Sstar, const double* Ps,
                 double h, int method, double* Pout, double* eT, int* iters);
void pmhd_residual_public(const orc_params& p, const Geom& G, const double* Ustar, double h,
                          const double* xg, double* E4, double* eT, double* eI);

}  // namespace orc
#endif
