/*
 * harmrad.h -- C ABI of the GB300 GRRMHD + M1 time-step library.
 *
 * The library advances the equations of general-relativistic radiation
 * magnetohydrodynamics with the M1 closure on a fixed Kerr-Schild or
 * Minkowski metric by one full time step, following Sec. 4 of McKinney,
 * Tchekhovskoy, Sadowski & Narayan (2014), "Three-dimensional GRRMHD
 * simulation of super-Eddington accretion, using a new code HARMRAD with M1
 * closure":
 *   - the RK3 method, same coefficients for explicit and implicit parts
 *     (Sec. 4.1, last paragraph);
 *   - per sub-step the algorithm of Sec. 4.2: ghost fill, U(P), geometric
 *     source, PPM/MC reconstruction (Sec. 4.3), face fluxes and wave speeds
 *     (Sec. 4.4), HLL or LAXF (Eqs. hll, lax), flux-CT EMFs, the update, and
 *     the implicit four-force solve (Sec. 4.7-4.11, Eq. source3) by a 4D
 *     Newton-Raphson (Eq. newton) with gas 1D_W (Sec. 4.5) and M1 (Sec. 4.6)
 *     inversions and back-ups.
 *
 * Units: c = G = M = 1, Heaviside-Lorentz magnetic field (Sec. 2).
 *
 * Primitive layout (12 FP64 values per zone, index order fixed):
 *   0 rho0  1 u_g  2-4 u~^i (ZAMO-relative gas 4-velocity, Sec. 2)
 *   5-7 B^i (lab-frame field)  8 Ebar (radiation-frame energy density)
 *   9-11 u~^i_rad (ZAMO-relative radiation-frame 4-velocity).
 * Conserved layout (densitised by sqrt(-g), Sec. 4 list of U_q):
 *   0 rho0 u^t  1 T^t_t + rho0 u^t  2-4 T^t_i  5-7 B^i  8 R^t_t  9-11 R^t_i.
 * Grid arrays exchanged through this API hold ACTIVE zones only, layout
 * [12][n3][n2][n1] with i (x1) fastest, contiguous FP64.
 *
 * Ownership and streams: the library owns all device state of a context.
 * Caller buffers are only read or written during the call, in order on the
 * CUDA stream given to harmrad_init (host buffers: the call returns after the
 * copy has completed).  Device pointers must be device memory of the current
 * device.  No call throws; every int-returning call reports through its return
 * code: 0 success, > 0 a warning, < 0 an error (see HARMRAD_E_*).
 */
#ifndef HARMRAD_H
#define HARMRAD_H

#ifdef __cplusplus
extern "C" {
#endif

#define HARMRAD_NPRIM 12

/* return codes */
#define HARMRAD_OK 0
#define HARMRAD_W_BACKUP_USED 1   /* some zones took the neighbour-average back-up */
#define HARMRAD_E_ARG (-1)        /* invalid argument or unsupported combination */
#define HARMRAD_E_CUDA (-2)       /* a CUDA runtime call failed */
#define HARMRAD_E_OOM (-3)        /* device allocation failed */
#define HARMRAD_E_NAN_INPUT (-4)  /* primitives given to set_prims are not finite */
#define HARMRAD_E_STATE (-5)      /* call out of order (e.g. step before set_prims) */

/* boundary conditions (bc[2*d] lower, bc[2*d+1] upper face of direction d) */
#define HARMRAD_BC_PERIODIC 0
#define HARMRAD_BC_OUTFLOW 1   /* copy the edge zone; the normal velocities may not point inward */
#define HARMRAD_BC_POLAR 2     /* theta direction of the Kerr-Schild grid only */
#define HARMRAD_BC_COPY 3      /* copy the edge zone (zero gradient), inflow allowed (shock tubes) */
#define HARMRAD_BC_FIXED 4     /* the ghost zones keep the values given by harmrad_set_prims_ghosts
                                  (a fixed inflow state, e.g. the base of the static atmosphere) */

#define HARMRAD_METRIC_MINKOWSKI 0
#define HARMRAD_METRIC_KS 1

#define HARMRAD_OPAC_CONST 0    /* kappa_abs = kappa_abs0 * rho0 (per length) */
#define HARMRAD_OPAC_KRAMERS 1  /* kappa_abs = kappa_abs0 * rho0^2 * max(T,T_min)^-3.5 */
#define HARMRAD_OPAC_FIELD 2    /* kappa_abs = kappa_scale * K, K a per-zone field
                                   (harmrad_set_opacity_field); ghosts follow the bc */
/* In every mode kappa_abs is multiplied by kappa_scale (also in FIELD mode,
 * above) and the scattering coefficient is kappa_scale * kappa_es0 * rho0;
 * both are per unit proper length. */

#define HARMRAD_RECON_PPM 0
#define HARMRAD_RECON_MC 1
#define HARMRAD_FLUX_LAXF 0
#define HARMRAD_FLUX_HLL 1

#define HARMRAD_PREC_FP64 0   /* every stage in FP64 */
#define HARMRAD_PREC_SPLIT 1  /* reconstruction, Riemann fluxes, EMFs in FP32 */

/* Time integrators (Sec. 4.1).  RK3 uses the same stages and coefficients for
 * the explicit and the implicit terms (the paper's runs: 3 sub-steps).  The
 * IMEX schemes are the paper's Eqs. IMEX2 (2 implicit stages and a final
 * combination: 3 sub-steps), IMEX2B (4 sub-steps) and IMEX3 (5 sub-steps);
 * their final combination has no implicit term, and its conserved state is
 * inverted by the same Newton solve with a zero source step.  A stage whose
 * explicit bracket holds no flux term runs no reconstruction or flux kernel. */
/* Gas equation of the implicit solve (Sec. 4.7, Eqs. source3-source6).
 * ENERGY: the energy-momentum equations, PMHD then URAD then PRAD; with RK3 a
 * zone that none of them solves (e_T > 1e-7) tries the entropy equation
 * (Eq. source6: [S u^t] - [S u^t]* = dt G_S, S = rho0 log(p^n/rho0^(n+1)),
 * Sec. 2) in place of the gas energy equation before the neighbour average
 * (Sec. 4.11); the radiation keeps total energy-momentum conservation.  The
 * entropy methods take the energy methods' sequence (PMHD, with u_g guessed
 * from the explicit entropy, then URAD and PRAD while e_T >= 1e-9); their
 * entropy row carries the factor T = p/rho0 and is normalised with the gas
 * energy row's norm added (Sec. 4.8).
 * ENTROPY: the entropy equation in every zone (same sequence; RK3 only), which
 * conserves the total entropy to round-off where the gas and radiation do not
 * exchange energy.  The entropy S u^t is carried as a 13th conserved quantity
 * with its own face fluxes (RK3 contexts).  A zone that neither the energy
 * nor the entropy equation solves tries the cold-MHD equations (Sec. 4.11)
 * when it is cold and momentum-dominated.  The point-wise entries
 * harmrad_zone_implicit and harmrad_zone_implicit_static have no explicit
 * entropy: the energy methods, then the cold-MHD equations;
 * harmrad_zone_implicit_full takes the entropy too. */
#define HARMRAD_EQ_ENERGY 0
#define HARMRAD_EQ_ENTROPY 1

/* Magnetic field transport (Sec. 4.2 steps viii-x).
 * FLUXCT: cell-centred B; the edge EMFs are the averages of the four face
 * fluxes of B around each edge and replace them (flux-CT, Toth 2000), which
 * keeps the corner-centred divergence of B at its initial value.
 * UCT: the paper's staggered field: sqrt(-g) B^d lives on the d-faces and is
 * advanced by the curl of edge EMFs from a 4-state upwind (HLL, or LAXF)
 * solution (Del Zanna et al. 2007): B^d of the faces interpolated to the edge
 * across d (MC-limited linear), the 3-velocities v^i = u^i/u^t of the four
 * cells around the edge extrapolated to it with MC-limited slopes, and signal
 * speeds averaged from the gas speeds of the two faces beside the edge.  The
 * face divergence sum_d (Bf_d(+) - Bf_d(-))/dx_d of every zone keeps its
 * initial value to round-off.  A zone's cell-centred B is the average of its
 * two faces' sqrt(-g) B^d over the centre's sqrt(-g).  harmrad_set_prims
 * initialises each face from the two cells beside it (and then the centres
 * from the faces); harmrad_set_face_fields sets the faces directly. */
#define HARMRAD_EMF_FLUXCT 0
#define HARMRAD_EMF_UCT 1

#define HARMRAD_INT_RK3 0
#define HARMRAD_INT_IMEX2 1
#define HARMRAD_INT_IMEX2B 2
#define HARMRAD_INT_IMEX3 3

/*
 * Run parameters.  Internal coordinates are uniform (Sec. 2): cell (i,j,k)
 * has centre x0 + (i+1/2) dx.  For the Kerr-Schild metric
 * r = R0 + exp(x1), theta = pi x2 + (1-hslope)/2 sin(2 pi x2), phi = 2 pi x3.
 * A direction with n = 1 is degenerate (no fluxes, no ghosts).
 */
typedef struct harmrad_params {
  int n[3];
  double x0[3], dx[3];
  int metric;
  double a_spin, R0, hslope;
  int bc[6];
  double gam;       /* adiabatic index of the gas, p = (gam-1) u_g */
  double a_rad;     /* radiation constant: Planck energy density a_rad T^4 */
  double courant;   /* Courant factor of the CFL time step (Sec. 4.4) */
  int opacity;
  double kappa_abs0, kappa_es0, kappa_scale, T_kappa_min;
  int recon, flux;
  double gamma_rad_max, gamma_gas_max;   /* Lorentz-factor caps (Sec. 4.6, 5) */
  double floor_rho0, floor_rho_pow, floor_u0, floor_u_pow;  /* floors f0 r^pow */
  double bsq_rho_max, bsq_u_max, u_rho_max;                 /* magnetisation caps */
  int newton_max;      /* Newton step limit per method (Sec. 4.10), <= 60 */
  double newton_tol;   /* PMHD tolerance on e_T (Sec. 4.10) */
  int precision;       /* HARMRAD_PREC_* */
  int integrator;      /* HARMRAD_INT_* */
  int implicit_eq;     /* HARMRAD_EQ_*: which gas equation the implicit solve uses */
  int emf;             /* HARMRAD_EMF_*: magnetic field transport */
} harmrad_params;

/* Per-zone outcome codes written by harmrad_get_status (worst over the
 * sub-steps of the last step).  Method sequence (Sec. 4.10): PMHD, then URAD,
 * then PRAD, the lowest-error solution kept; a zone whose radiation is
 * extremely sub-dominant (below 10 eps_m of the gas in conserved or
 * fluid-frame energy) starts with URAD and skips PMHD. */
#define HARMRAD_ZONE_PMHD 0    /* PMHD Newton accepted */
#define HARMRAD_ZONE_URAD 1    /* a retry method (URAD, PRAD, the entropy or the cold-MHD
                                  equations) gave the accepted solution */
#define HARMRAD_ZONE_BACKUP 2  /* no method reached e_T <= 1e-7: neighbour average */

typedef struct harmrad_stats {
  double dt;                   /* time step used by the last harmrad_step */
  long long zone_stages;       /* implicit solves in the last step */
  long long pmhd_ok, urad_ok, backup;
  long long newton_iters;      /* Newton steps summed over all solves */
  int kernel_launches;         /* kernels one harmrad_step launches */
  int graph;                   /* 1 if the step is replayed as a CUDA graph */
  long long entropy_ok;        /* solves whose accepted solution came from the entropy
                                  equation (counted in urad_ok as well, or in pmhd_ok with
                                  implicit_eq = 1) */
  long long cold_ok;           /* solves whose accepted solution came from the cold-MHD
                                  equations (counted in urad_ok as well); their u_g is the
                                  neighbours' average */
} harmrad_stats;

typedef struct harmrad_ctx harmrad_ctx;

/* Allocate a context for one grid on the current device.  stream: a
 * cudaStream_t (NULL = legacy default stream).  Returns HARMRAD_E_ARG for
 * invalid parameters (non-positive sizes, POLAR on a non-theta face or with
 * an odd n3 > 1, newton_max outside [1,60], ...), HARMRAD_E_OOM when device
 * memory is exhausted. */
int harmrad_init(const harmrad_params* p, void* stream, harmrad_ctx** out);

/* Allocate one context for a batch of count independent grids ("boxes"),
 * advanced together: every kernel of a step covers all boxes, so a batch of
 * small boxes runs in the launches one grid takes.  p[0..count-1] may differ
 * only in n, x0, dx and bc; the active directions (n > 1) and every physics
 * parameter must agree (HARMRAD_E_ARG otherwise).  Arrays exchanged with the
 * context (primitives, status, iterations, opacity field) hold the boxes'
 * active-zone blocks one after another, box 0 first, each in the single-grid
 * layout.  Each box takes its own CFL time step when harmrad_step gets dt <= 0
 * (the boxes are independent problems); harmrad_cfl_dt and harmrad_stats.dt
 * report the smallest.  harmrad_init(p, s, out) is harmrad_init_batch(p, 1, s,
 * out).  harmrad_compute_fluxes accepts single-grid contexts only. */
int harmrad_init_batch(const harmrad_params* p, int count, void* stream, harmrad_ctx** out);

/* Release all device state of the context (NULL is ignored). */
void harmrad_destroy(harmrad_ctx* ctx);

/* Load the active-zone primitives ([12][n3][n2][n1] FP64).  on_device != 0:
 * P is a device pointer, else host memory.  Returns HARMRAD_E_NAN_INPUT if any
 * value is not finite, or if rho0, u_g or Ebar is not positive. */
int harmrad_set_prims(harmrad_ctx* ctx, const double* P, int on_device);

/* Load the primitives of every cell of a single-grid context, ghost zones
 * included: layout [12][N3][N2][N1] with N_d = n_d + 8 for an active
 * direction (4 ghosts per side) and N_d = 1 for a degenerate one.  The ghost
 * zones of faces with HARMRAD_BC_FIXED keep these values through every later
 * step (the fixed boundary states of the paper's static atmosphere, Sec. 5);
 * all other ghosts are refilled by their boundary condition at every
 * sub-step.  A later harmrad_set_prims changes the active zones only.
 * HARMRAD_E_ARG for a batch; HARMRAD_E_NAN_INPUT as for harmrad_set_prims,
 * over every cell. */
int harmrad_set_prims_ghosts(harmrad_ctx* ctx, const double* P, int on_device);

/* Staggered field (HARMRAD_EMF_UCT contexts of one grid; HARMRAD_E_ARG
 * otherwise): sqrt(-g) B^d on the d-faces, three arrays one after another,
 * direction d of shape [n3'][n2'][n1'] (FP64) with n_d' = n_d + 1 faces along
 * d when n_d > 1 (1 otherwise) and n_e' = n_e across.  On a periodic
 * direction the last face is the image of the first: set ignores it, get
 * returns the image.  Set makes the cell-centred B of every zone the average
 * of its faces; call it after harmrad_set_prims (which initialises the faces
 * from the cell-centred B). */
int harmrad_set_face_fields(harmrad_ctx* ctx, const double* Bf, int on_device);
int harmrad_get_face_fields(harmrad_ctx* ctx, double* Bf, int on_device);

/* Load the per-zone absorption field K (active zones, [n3][n2][n1] FP64 per
 * box, boxes concatenated) of a context created with opacity =
 * HARMRAD_OPAC_FIELD (HARMRAD_E_ARG otherwise); kappa_abs = kappa_scale * K per
 * unit length.  Ghost values follow the boundary conditions like the
 * primitives.  Returns HARMRAD_E_NAN_INPUT for a negative or non-finite value.
 * The field starts at zero; it is kept until the next call. */
int harmrad_set_opacity_field(harmrad_ctx* ctx, const double* K, int on_device);

/* Copy the active-zone primitives out (same layout). */
int harmrad_get_prims(harmrad_ctx* ctx, double* P, int on_device);

/* CFL time step of the current state: Courant factor times the minimum over
 * zones of 1 / sum_d (v_d / dx_d), v_d the largest gas or radiation signal
 * speed on the two d-faces of the zone (Sec. 4.4, last paragraph). */
int harmrad_cfl_dt(harmrad_ctx* ctx, double* dt);

/* Advance one full step of the context's integrator (RK3 or an IMEX scheme).
 * dt <= 0 selects the CFL step of the current
 * state (computed on the device).  The call only enqueues work on the
 * context's stream and does not wait for it; solver outcomes (back-up use,
 * iteration counts) are read afterwards with harmrad_get_stats. */
int harmrad_step(harmrad_ctx* ctx, double dt);

/* Advance one full step with host input and output: copies P_in (host,
 * active zones) to the device, steps with dt (<= 0: CFL), copies the result to
 * P_out (host).  P_in and P_out may alias. */
int harmrad_step_host(harmrad_ctx* ctx, const double* P_in, double* P_out, double dt);

/* Solver statistics of the last step (synchronises the stream).  Returns
 * HARMRAD_W_BACKUP_USED if any zone took the neighbour-average back-up. */
int harmrad_get_stats(harmrad_ctx* ctx, harmrad_stats* st);

/* Per-zone outcome bytes of the last step ([n3][n2][n1]). */
int harmrad_get_status(harmrad_ctx* ctx, unsigned char* st, int on_device);

/* Per-zone Newton iteration totals of the last step ([n3][n2][n1] int32). */
int harmrad_get_iters(harmrad_ctx* ctx, int* it, int on_device);

/* Face fluxes of direction dir (1..3) for the current primitives after ghost
 * fill, reconstruction, Riemann solve and flux-CT, as the first sub-step of a
 * step would compute them; layout [12][n3'][n2'][n1'] with n_dir' = n_dir + 1
 * (faces 0..n_dir), FP64, host memory.  Diagnostic for tests. */
int harmrad_compute_fluxes(harmrad_ctx* ctx, int dir, double* F_host);

/* Point-wise physics at n independent points (device pointers, row-major;
 * opacity mode HARMRAD_OPAC_FIELD is rejected with HARMRAD_E_ARG):
 * x[n][4] internal coordinates, P[n][12] primitives ->
 * U[n][12] conserved, SM[n][12] geometric source, F[n][3][12] fluxes,
 * speeds[n][3][4] (gas vmin, vmax, rad vmin, vmax per direction).  Any output
 * pointer may be NULL. */
int harmrad_zone_physics(const harmrad_params* p, int n, const double* x, const double* P,
                         double* U, double* SM, double* F, double* speeds, void* stream);

/* Method codes of the zone-level solves below: HARMRAD_ZONE_PMHD,
 * HARMRAD_ZONE_URAD (URAD or PRAD) and HARMRAD_ZONE_BACKUP (no method reached
 * e_T <= 1e-7; Pout holds the guess with B of U*), and, for the back-up
 * equations of Sec. 4.11: */
#define HARMRAD_ZONE_ENTROPY 3 /* the entropy equation (Eq. source6) in place of the energy equation */
#define HARMRAD_ZONE_COLD 4    /* the cold-MHD equations: momentum only, u_g held at the guess */

/* Implicit four-force solve of n independent zones (device pointers):
 * x[n][4], Ustar[n][12] explicit conserved state, Ps[n][12] guess primitives,
 * h[n] = b_s dt -> Pout[n][12], eT[n], iters[n], method[n] (the codes above).
 * Same solver and method sequence as harmrad_step (Sec. 4.7-4.11) without the
 * explicit entropy: PMHD, URAD, PRAD, then the cold-MHD equations for a cold,
 * momentum-dominated zone.  The grid step then replaces a cold-MHD zone's u_g
 * by its neighbours' average; a single zone has no neighbours, so Pout keeps
 * the solve's u_g (the guess's). */
int harmrad_zone_implicit(const harmrad_params* p, int n, const double* x, const double* Ustar,
                          const double* Ps, const double* h, double* Pout, double* eT, int* iters,
                          unsigned char* method, void* stream);

/* As harmrad_zone_implicit with the explicit entropy Sstar[n] (device, may be
 * NULL) = sqrt(-g) S u^t of the zone after the explicit update, S u^t =
 * rho0 u^t s_gas (Sec. 2, Eq. S): a zone that the energy methods leave without
 * a solution tries the entropy equation (HARMRAD_ZONE_ENTROPY) before the
 * cold-MHD equations, as in harmrad_step's RK3 stages.  A non-finite Sstar[i]
 * skips the entropy equation for that zone. */
int harmrad_zone_implicit_full(const harmrad_params* p, int n, const double* x, const double* Ustar,
                               const double* Sstar, const double* Ps, const double* h, double* Pout,
                               double* eT, int* iters, unsigned char* method, void* stream);

/* One Newton method of the implicit solve alone on n independent zones
 * (device pointers; for testing each method against its restatement):
 * method 0 PMHD from the gas of Ps, 1 URAD from R^t_nu of Ps, 2 PRAD from the
 * radiation of Ps (Sec. 4.8-4.10), 3 the staged PMHD of Sec. 4.10 (one
 * momentum-only step damped by 1/2, energy-only steps, then the full 4D
 * Newton with its first step damped by 1/4, two-sided differences) from the
 * gas of Ps with u_g from the explicit entropy Sstar (device, may be NULL),
 * 4 the staged URAD and 5 the staged PRAD (the same stages on the radiation
 * unknowns with the plain methods' one-sided differences; guesses as 1, 2),
 * 6, 7, 8 the entropy-based PMHD, URAD, PRAD (the entropy equation, Eq.
 * source6, in place of the energy equation with Sstar, which these require;
 * guesses as 0, 1, 2).
 * Pout[n][12]: the best iterate's primitives as its error function forms them
 * (radiation through the TYPE2 limiter; Ps where no residual was finite),
 * eT[n] its total error (inf if none), iters[n] the Newton steps.
 * HARMRAD_E_ARG for another method or a per-zone opacity field. */
int harmrad_zone_method(const harmrad_params* p, int n, const double* x, const double* Ustar,
                        const double* Sstar, const double* Ps, const double* h, int method, double* Pout,
                        double* eT, int* iters, void* stream);

/* Same solve as harmrad_zone_implicit, for callers that cannot allocate device
 * memory: processes whose device memory is owned by another allocator (a
 * framework's caching pool, a fixed-budget service) and may not call
 * cudaMalloc or cudaFree, whose implicit synchronisation they also cannot
 * afford.  The paper has no counterpart; this is a deployment variant.
 * The zones that PMHD does not accept are queued for URAD/PRAD in a fixed array in
 * the library's static device memory (about 2.9 MB per device that loads the
 * library, kept until the process exits); the call makes no device
 * allocation.  n must not exceed 65536 (HARMRAD_E_ARG otherwise).  The first
 * call on a device looks up that array's device address, so make it before
 * any stream capture; the address is kept per device together with the id of
 * the CUDA context it belongs to, and looked up again by the first call in a
 * new context (after a device reset).  The array is shared by every call on the device and
 * keeps the last call's contents (each call clears its queue counter first):
 * calls whose work overlaps on the GPU race, so serialise them, e.g. on one
 * stream.  Arguments, layouts and outputs as for harmrad_zone_implicit; the
 * call synchronises the stream before returning. */
int harmrad_zone_implicit_static(const harmrad_params* p, int n, const double* x,
                                 const double* Ustar, const double* Ps, const double* h,
                                 double* Pout, double* eT, int* iters, unsigned char* method,
                                 void* stream);

/* Kernel classes timed by harmrad_profile_step. */
#define HARMRAD_K_BC 0        /* ghost-zone fill */
#define HARMRAD_K_PREP 1      /* per-cell metric factors and flattener inputs */
#define HARMRAD_K_FLATTEN 2   /* PPM shock flattener */
#define HARMRAD_K_FACE 3      /* face physics + Riemann flux */
#define HARMRAD_K_CT 4        /* flux-CT EMFs */
#define HARMRAD_K_UPDATE 5    /* update + geometric source + PMHD implicit solve */
#define HARMRAD_K_RETRY 6     /* retry queue (URAD, PRAD) */
#define HARMRAD_K_BACKUP 7    /* neighbour-average back-up */
#define HARMRAD_K_CFL 8       /* CFL reduction */
#define HARMRAD_K_OTHER 9     /* memsets, time-step upload */
#define HARMRAD_K_EDGE 10     /* PPM / MC reconstruction of the face values */
#define HARMRAD_K_CLASSES 11

typedef struct harmrad_kernel_times {
  double ms[HARMRAD_K_CLASSES];  /* summed device time per class, milliseconds */
  int launches[HARMRAD_K_CLASSES];
  int total_launches;
} harmrad_kernel_times;

/* Advance one full step like harmrad_step, launched without the CUDA graph and
 * with a CUDA event recorded after every kernel on the context's stream; the
 * time between consecutive events is summed per kernel class.  Synchronises
 * the stream.  For benchmarking and profiling. */
int harmrad_profile_step(harmrad_ctx* ctx, double dt, harmrad_kernel_times* out);

/* Adjoint of the step (reverse-mode derivative), FP64 single-grid contexts.
 *
 * harmrad_adjoint_enable(ctx, 1) allocates the adjoint's workspace (about 40
 * doubles per cell) and makes every later harmrad_step keep a copy of its
 * input; 0 releases it.  HARMRAD_E_ARG for a batch, split precision or an
 * IMEX integrator, or a context with a HARMRAD_BC_FIXED face.
 *
 * harmrad_step_adjoint(ctx, gP_out, gP_in, g_kappa, on_device) differentiates
 * the last harmrad_step of the context: given gP_out = dL/dP^{n+1} (active
 * layout [12][n3][n2][n1]) it writes gP_in = dL/dP^n (same layout; may alias
 * gP_out) and *g_kappa = dL/d kappa_scale (g_kappa may be NULL), with the time
 * step of that step held fixed.  It recomputes the step from the saved input
 * (the context's primitives end as that step's result again) and sweeps the
 * three sub-steps in reverse: implicit solve by the implicit-function theorem
 * at the converged solution (one transposed 4x4 solve per zone, no unrolled
 * Newton iterations), explicit update, flux-CT, Riemann fluxes,
 * reconstruction, flattener, ghost fill, each as the transpose of its local
 * Jacobian.  Branches (limiters, wave-speed maxima, flattener clamps, outflow
 * clamps) take the derivative of the branch the step took.  Zones whose
 * solution a floor changed are constant except for B; back-up zones pass
 * their cotangent to the neighbours they averaged.  Zones solved by the
 * entropy equation (by its PMHD, URAD or PRAD, which solve the same
 * equations) take the transposed solve of that system.  The paper has
 * no adjoint; this is an extension.  HARMRAD_E_STATE if no step ran since
 * enabling; HARMRAD_E_ARG if a zone of the step was solved by the cold-MHD
 * equations (its u_g, the neighbours' average, has no adjoint here). */
int harmrad_adjoint_enable(harmrad_ctx* ctx, int on);
int harmrad_step_adjoint(harmrad_ctx* ctx, const double* gP_out, double* gP_in, double* g_kappa,
                         int on_device);

/* Branch signature, an instrument for derivative checks (the paper has none):
 * a finite difference (L(P + h v) - L(P - h v)) / 2h measures the derivative
 * only if the step takes the same branches at P + h v and at P - h v.  With
 * the signature on, every later step folds each branch decision it takes into
 * a 64-bit word of the cell concerned: the MC slope limiter's choice per
 * primitive and direction, the PPM monotonicity limiter's case, the shock
 * flattener's tests and clamps and the maxima it takes, the wave-speed maxima
 * of LAXF/HLL and the speed caps of both states at every face, the outflow
 * clamps of the ghost fill, the floors that act, the TYPE2 limiter and the
 * solver method of every zone, and the neighbours a back-up averages; each
 * decision is hashed with its kernel and sub-step and the words combine by
 * XOR.  Two runs from different states took the same branches everywhere if
 * and only if their words agree (up to 64-bit hash collisions).
 * harmrad_branch_signature(ctx, 1) allocates the words (one per cell of the
 * ghost-inclusive grid, [N3][N2][N1] per grid) and sets them to zero; 0 frees
 * them.  Drops the captured graphs.  The decisions add no arithmetic to the
 * step's results. */
int harmrad_branch_signature(harmrad_ctx* ctx, int on);
/* Copy the signature words out (host or device memory; ncell values).
 * HARMRAD_E_STATE if the signature is off.  Synchronises the stream. */
int harmrad_get_branch_signature(harmrad_ctx* ctx, unsigned long long* out, int on_device);

/* Make P (active layout, host or device per on_device) with time step dt > 0
 * the step that the next harmrad_step_adjoint differentiates, without running
 * that step: P becomes the context's primitives and the adjoint's saved input,
 * exactly as harmrad_step(ctx, dt) from P would record them (the adjoint
 * recomputes the step itself).  For checkpointed reverse sweeps that already
 * hold every step's input.  HARMRAD_E_STATE unless the adjoint is enabled,
 * HARMRAD_E_ARG for dt <= 0; HARMRAD_E_NAN_INPUT as for harmrad_set_prims. */
int harmrad_adjoint_set_input(harmrad_ctx* ctx, const double* P, double dt, int on_device);

/* Launch shapes of the three heaviest kernels: threads per block and the cap
 * on blocks per SM of their grid-stride grids (the grid is the smaller of the
 * work and sms x cap blocks).  Shapes change no result: every zone and face
 * runs the same arithmetic under any shape. */
typedef struct harmrad_tuning {
  int face_block, face_blocks_per_sm;      /* face physics + Riemann; block 32..128 */
  int update_block, update_blocks_per_sm;  /* update + implicit solve; block 32..128 */
  int edge_block, edge_blocks_per_sm;      /* reconstruction; block 32..256 */
  int newton_split;  /* PMHD iterations the update kernel runs before a zone moves to the
                        compacted continuation queue (0: none, the zone finishes in place);
                        1..60.  The resumed iteration is the same arithmetic. */
  double face_ms, update_ms, edge_ms;      /* autotune: best device ms per step */
} harmrad_tuning;

/* Autotune the launch shapes on the context's current state: time `reps`
 * eager steps (dt <= 0: CFL) for each candidate shape, with CUDA events on the
 * context's stream, keep the fastest per kernel class, restore the primitives
 * and drop the captured graphs (the next step re-captures).  Candidates:
 * blocks of 64 or 128 threads (edges 128 or 256) with caps of 4..64 blocks per
 * SM, and Newton splits of 0 (no continuation queue), 3 and 5.  Writes the chosen shapes to *out (may be NULL).  Synchronises; allocates
 * a scratch copy of the primitives for the duration of the call. */
int harmrad_autotune(harmrad_ctx* ctx, int reps, harmrad_tuning* out);

/* Read or set the launch shapes (set: values outside the ranges above give
 * HARMRAD_E_ARG; the captured graphs are dropped). */
int harmrad_get_tuning(harmrad_ctx* ctx, harmrad_tuning* out);
int harmrad_set_tuning(harmrad_ctx* ctx, const harmrad_tuning* t);

/* FP64 fused multiply-add rate of the current device in TFLOP/s (2 flops per
 * FMA), measured on the given stream by a kernel of independent FMA chains
 * (8 per thread, 8 blocks of 256 threads per SM, 4096 rounds): the best of
 * reps timed launches after one warm-up, CUDA events around each.  It is the
 * FP64 peak that the roofline fraction of the FP64-bound kernels divides by;
 * no step of the method uses it.  Allocates and frees a small scratch buffer;
 * synchronises the stream.  HARMRAD_E_ARG unless 1 <= reps <= 100. */
int harmrad_fp64_fma_rate(int reps, double* tflops, void* stream);

/* Human-readable text of a return code. */
const char* harmrad_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HARMRAD_H */
