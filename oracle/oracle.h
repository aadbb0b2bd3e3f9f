/*
 * HARMRAD oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of one GRRMHD+M1 time step of
 * McKinney, Tchekhovskoy, Sadowski & Narayan (2014), "Three-dimensional
 * GRRMHD simulation of super-Eddington accretion, using a new code HARMRAD
 * with M1 closure".  It exists only so that tests, the smoke check and the
 * benchmark's CPU-baseline leg can check and time the CUDA library against an
 * independent implementation.  It shares no code, header or constant table
 * with the CUDA path, and nothing in the product may call it.
 *
 * Conventions (paper Sec. 2-4): c = G = M = 1, Heaviside-Lorentz B.
 * Primitive vector P (12 doubles per zone, index order fixed below):
 *   rho0, u_g, u~^1..3 (ZAMO-relative gas 4-velocity), B^1..3 (lab field),
 *   Ebar (radiation-frame energy density), u~^1..3_rad.
 * Conserved vector U (densitised by sqrt(-g)):
 *   rho0 u^t, T^t_t + rho0 u^t, T^t_i, B^i, R^t_t, R^t_i.
 * Arrays passed through this API hold active zones only, layout
 * [12][n3][n2][n1] (i fastest).
 *
 * Pinned by tests/test_oracle_pins.py (closed forms, textbook SR-MHD, M1
 * closure identities, exact scalar roots, conservation) and by
 * tests/test_oracle_waves.py (the linear-wave eigenvalues the paper prints in
 * its Table t.waves: wave speed and radiative damping of sound, fast and slow
 * modes, optically thin and thick, gas- and radiation-dominated), by
 * tests/test_oracle_shocks.py (the jump conditions of the radiative shock-tube
 * states of Table t.radtube) and by tests/test_oracle_imex.py (the orders of
 * accuracy of the IMEX integrators on stiff relaxation).  The readings of
 * the paper where it points to sources that are not in it are pinned by
 * tests/test_oracle_readings.py: the polar-axis ghost rule (a smooth
 * Cartesian field continued across the axis), the floors (the bounds they
 * establish, the velocity and field they keep, idempotence), the PPM edge
 * values (exact for a parabola, fourth order on smooth data, a monotone
 * limited parabola) and the Kerr-Schild signal speeds (velocity addition in
 * the normal observer's frame).  Parity unpinned: the constants of the PPM
 * shock flattener beyond SP0 = 0.75 (not in the paper), which only
 * oracle-versus-library agreement checks.
 */
#ifndef HARMRAD_ORACLE_H
#define HARMRAD_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n[3];               /* active zones per direction (1 = degenerate) */
  double x0[3], dx[3];    /* uniform internal coordinates of the lower edge */
  int metric;             /* 0 Minkowski Cartesian, 1 Kerr-Schild + MSP map */
  double a_spin, R0, hslope;
  int bc[6];              /* lower/upper per direction: 0 periodic, 1 outflow, 2 polar,
                             3 zero gradient with inflow allowed, 4 fixed (ghosts as set
                             by orc_set_prims_with_ghosts) */
  double gam, a_rad, courant;
  int opacity;            /* 0 kappa = k0*rho (per length), 1 Kramers k0*rho^2*T^-3.5,
                             2 per-zone field K (orc_set_opacity_field), kappa = K */
  double kappa_abs0, kappa_es0, kappa_scale, T_kappa_min;
  int recon;              /* 0 PPM, 1 MC */
  int flux;               /* 0 LAXF, 1 HLL */
  double gamma_rad_max, gamma_gas_max;
  double floor_rho0, floor_rho_pow, floor_u0, floor_u_pow;
  double bsq_rho_max, bsq_u_max, u_rho_max;
  int newton_max;
  double newton_tol;
  int integrator;         /* 0 RK3 with the same coefficients for the explicit and
                             implicit parts (the paper's runs), 1 IMEX2, 2 IMEX2B,
                             3 IMEX3 (Sec. 4.1, Eqs. IMEX2, IMEX2B, IMEX3) */
  int implicit_eq;        /* 0 energy equations, the entropy equation as back-up (RK3);
                             1 the entropy equation in every zone (RK3) */
  int emf;                /* 0 flux-CT: cell-centred B, edge EMFs averaged from the face
                             fluxes; 1 staggered B on faces with the 4-state upwind EMF
                             (Sec. 4.2 steps viii-ix) */
} orc_params;

/* Per-zone solver outcome codes (same meaning as the library's status byte). */
enum { ORC_OK_PMHD = 0, ORC_OK_URAD = 1, ORC_BACKUP = 2 };

typedef struct {
  double e_T;      /* total normalised error of the accepted solution */
  int iters_pmhd;  /* Newton iterations taken by the PMHD attempt */
  int iters_urad;  /* Newton iterations taken by the URAD attempt (0 if none) */
  int method;      /* ORC_OK_PMHD, ORC_OK_URAD or ORC_BACKUP */
  int neg_erad;    /* 1 if the accepted solution hit the TYPE2 negative-energy branch */
  int entropy;     /* 1 if the entropy equation gave the accepted solution */
  int cold;        /* 1 if the cold-MHD equations gave it (u_g held at the guess) */
} orc_implicit_info;

/* --- grid-level driver --------------------------------------------------- */
void*  orc_create(const orc_params* p);
void   orc_destroy(void* ctx);
void   orc_set_prims(void* ctx, const double* P);
void   orc_get_prims(void* ctx, double* P);
/* Absorption field K of opacity mode 2, active zones [n3][n2][n1]; absorption
 * per unit length kappa_scale * K; ghosts follow the boundary conditions. */
void   orc_set_opacity_field(void* ctx, const double* K);
double orc_cfl_dt(void* ctx);
/* One full RK3 step; dt <= 0 means use the CFL time step. Returns the dt used. */
double orc_step(void* ctx, double dt);
/* Per-zone status bytes of the last step, worst over its three stages ([n3][n2][n1]). */
void   orc_get_status(void* ctx, unsigned char* st);
/* Staggered field (emf = 1): sqrt(-g) B^d on the d-faces, three arrays one
 * after another, direction d of shape [n3'][n2'][n1'] with n_d' = n_d + 1
 * faces along d when n_d > 1 (1 otherwise) and n_e' = n_e across.  On a
 * periodic direction the last face is the first one's image: set ignores it,
 * get returns the image.  Set also makes the cell-centred B of every active
 * zone the average of its two faces (sqrt(-g) B averaged). */
void   orc_set_face_fields(void* ctx, const double* Bf);
void   orc_get_face_fields(void* ctx, double* Bf);
/* Per-zone Newton iteration totals summed over the three stages of the last step. */
void   orc_get_iters(void* ctx, int* it);
/* Counts over the last step: [0] PMHD-accepted, [1] URAD-accepted, [2] back-up,
 * [3] total Newton iterations, [4] zone-stages solved, [5] zone-stages whose
 * accepted solution came from the entropy equation, [6] from the cold-MHD
 * equations. */
void   orc_get_counts(void* ctx, long long* c);
/* Face fluxes of one direction after the last call to orc_compute_fluxes
 * (debug/test hook): computes ghost fill + fluxes (+flux-CT) for the current
 * prims and copies F for faces [0..n_d] x active transverse range,
 * layout [12][n3'][n2'][n1'] where n_d' = n_d + 1. */
void   orc_compute_fluxes(void* ctx, int dir, double* F);
/* Set every cell, ghosts included (layout [12][N3][N2][N1], N = n + 8 for an
 * active direction); ghosts of fixed faces (bc 4) keep these values. */
void   orc_set_prims_with_ghosts(void* ctx, const double* P);
/* Ghost-inclusive prim copy (layout [12][N3][N2][N1]); debug/test hook. */
void   orc_get_prims_with_ghosts(void* ctx, double* P, int fill_ghosts);

/* --- point-wise physics (for pins) --------------------------------------- */
/* Metric at internal coordinates x[4] = (t, x1, x2, x3). */
void   orc_metric(const orc_params* p, const double* x, double* gcov16,
                  double* gcon16, double* gdet, double* alpha);
/* Connection Gamma^l_{m k} at x, layout [l][m][k]. */
void   orc_connection(const orc_params* p, const double* x, double* gam64);
/* U(P) and geometric source SM(P) at x (12 each). */
void   orc_prim_to_cons(const orc_params* p, const double* x, const double* P,
                        double* U, double* SM);
/* Flux along direction d (1..3) at x, plus gas and radiation wave speeds
 * (vmin,vmax)[gas], (vmin,vmax)[rad]. */
void   orc_flux(const orc_params* p, const double* x, int d, const double* P,
                double* F, double* speeds4);
/* Full mixed stress tensors T^mu_nu and R^mu_nu ([mu][nu], 16 each). */
void   orc_stress(const orc_params* p, const double* x, const double* P,
                  double* T16, double* R16);
/* Covariant four-force G_nu (Eq. Gcov) for prims P at x. */
void   orc_four_force(const orc_params* p, const double* x, const double* P,
                      double* G4);
/* M1 inversion from R^t_nu (4) to (Ebar, u~^i_rad) (4). limiter: 0 BASIC, 2 TYPE2.
 * Returns 1 if the limiter saw E_rad <= 0. */
int    orc_rad_invert(const orc_params* p, const double* x, const double* Rt,
                      int limiter, double* Prad);
/* Gas 1D_W inversion from U (12, densitised) using guess prims Pg (12);
 * writes prims 0..4 of Pout and copies B. Returns 0 on success. */
int    orc_gas_invert(const orc_params* p, const double* x, const double* U,
                      const double* Pg, double tol, double* Pout);
/* Sec. 4.10 sub-dominance test of one zone: 1 if the radiation is extremely
 * sub-dominant (URAD first in the grid step). */
int    orc_radiation_subdominant(const orc_params* p, const double* x, const double* Ustar,
                                 const double* Ps);
/* Sec. 4.11 test of one zone for the cold-MHD back-up: 1 if the guess Ps is
 * cold (u_g < 0.1 rho0 u~^i u~_i) and both the gas t^t_mu and the radiation
 * R^t_mu of U* are momentum-dominated (|t_t t^t| < 0.1 |t_i t^i|). */
int    orc_cold_allowed(const orc_params* p, const double* x, const double* Ustar, const double* Ps);
/* Implicit four-force solve of one zone: U* (12, densitised), the explicit
 * entropy S* = sqrt(-g) S u^t (NULL: no entropy back-up), guess P_s,
 * h = b_s*dt, the grid step's method sequence.  Writes the new prims and info. */
void   orc_implicit_zone(const orc_params* p, const double* x, const double* Ustar,
                         const double* Sstar, const double* Ps, double h, double* Pout,
                         orc_implicit_info* info);
/* One Newton method alone on one zone (test hook): method 0 PMHD (guess the
 * gas of Ps), 1 URAD (guess R^t_nu of Ps), 2 PRAD (guess the radiation of Ps),
 * 3 staged PMHD (Sec. 4.10; guess the gas of Ps with u_g from the explicit
 * entropy Sstar = sqrt(-g) S u^t when Sstar is not NULL), 4 staged URAD,
 * 5 staged PRAD (guesses as 1 and 2), 6, 7, 8 the entropy-based PMHD, URAD,
 * PRAD (Eq. source6 with the explicit entropy Sstar; guesses as 0, 1, 2).
 * Writes the best
 * iterate's prims (Ps if none), its e_T (inf if none) and the Newton steps
 * taken. */
void   orc_method_zone(const orc_params* p, const double* x, const double* Ustar,
                       const double* Sstar, const double* Ps, double h, int method,
                       double* Pout, double* eT, int* iters);
/* Residual of the PMHD system at gas unknowns xg = (u_g, u~^i):
 * E[4] (gas rows), eT, eI.  Test hook. */
void   orc_pmhd_residual(const orc_params* p, const double* x, const double* Ustar,
                         double h, const double* xg, double* E4, double* eT,
                         double* eI);
/* Face flux of direction d (1..3) from an 8-cell stencil S[8][12] of active or
 * ghost primitives along d (cells f-4 .. f+3 around the face f), with the
 * stencil cells' internal coordinates xc[8][3] and the face centre xf[3];
 * fresh flattener (first sub-step), no flux-CT.  Writes F[12] and the face's
 * max signal speed.  Test hook for sampled faces of large grids. */
void   orc_face_flux_stencil(const orc_params* p, int d, const double* S, const double* xc,
                             const double* xf, double* F, double* speed);
/* Floors of the grid step applied to the primitives P (12, in place) of a
 * zone at x (test hook). */
void   orc_apply_floors(const orc_params* p, const double* x, double* P);
/* PPM reconstruction of the centre cell of the 5-cell stencil s5 (Sec. 4.3):
 * edge values aL, aR with flattener chi (test hook). */
void   orc_ppm_cell(const double* s5, double chi, double* aL, double* aR);
/* Monotonised-central slope of the centre cell (test hook). */
double orc_mc_slope(double qm, double q0, double qp);
/* Levermore Eddington factor xi(f) (Sec. 3.1). */
double orc_levermore_xi(double f);

#ifdef __cplusplus
}
#endif
#endif
