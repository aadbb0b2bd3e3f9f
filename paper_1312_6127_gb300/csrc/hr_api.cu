// C ABI of the harmrad library: context management, data movement and the
// sequence of one full RK3 step (Sec. 4.1-4.2 of McKinney et al. 2014),
// replayed as a CUDA graph.  A context holds one grid, or the boxes of a
// batch, all advanced by the same kernel launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hr_adjoint.cuh"
#include "hr_ctx.h"
#include "hr_uct.cuh"

using hr::BoxGeo;
using hr::DevParams;

namespace {

#define HR_CHECK(x)                          \
  do {                                       \
    if ((x) != cudaSuccess) {                \
      cudaGetLastError();                    \
      return HARMRAD_E_CUDA;                 \
    }                                        \
  } while (0)

// Active layout of a context: the grids' [nv][n3][n2][n1] blocks one after the
// other.  These kernels move nv planes between it and the ghost-inclusive
// cell layout (nv = 12 for the primitives, 1 for the opacity field).
__global__ void k_unpack(const BoxGeo* __restrict__ boxes, int nbox, int nv,
                         const double* __restrict__ src, double* __restrict__ dst0) {
  for (int b = 0; b < nbox; ++b) {
    const BoxGeo bx = boxes[b];
    const double* s = src + nv * bx.aoff;
    double* dst = dst0 + nv * bx.coff;
    long long total = (long long)nv * bx.nact;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
      long long q = id / bx.nact, z = id % bx.nact, r = z;
      int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      int j = (int)(r % bx.n[1]);
      int k = (int)(r / bx.n[1]);
      dst[q * bx.ntot + hr::cell_index(bx, i, j, k)] = s[id];
    }
  }
}

__global__ void k_pack(const BoxGeo* __restrict__ boxes, int nbox, const double* __restrict__ P0,
                       double* __restrict__ dst0) {
  for (int b = 0; b < nbox; ++b) {
    const BoxGeo bx = boxes[b];
    const double* P = P0 + 12 * bx.coff;
    double* d = dst0 + 12 * bx.aoff;
    long long total = (long long)hr::NPR * bx.nact;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
      long long q = id / bx.nact, z = id % bx.nact, r = z;
      int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      int j = (int)(r % bx.n[1]);
      int k = (int)(r / bx.n[1]);
      d[id] = P[q * bx.ntot + hr::cell_index(bx, i, j, k)];
    }
  }
}

// flag = 1 if any value is not finite or rho0, u_g, Ebar is not positive
// (nv = 12), or if any opacity-field value is negative or not finite (nv = 1)
__global__ void k_validate(const BoxGeo* __restrict__ boxes, int nbox, int nv,
                           const double* __restrict__ src, int* flag) {
  for (int b = 0; b < nbox; ++b) {
    const BoxGeo bx = boxes[b];
    const double* s = src + nv * bx.aoff;
    long long total = (long long)nv * bx.nact;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
      double v = s[id];
      long long q = id / bx.nact;
      bool bad = !isfinite(v);
      if (nv == 12) bad = bad || ((q == hr::RHO || q == hr::UU || q == hr::ER) && !(v > 0.0));
      else bad = bad || v < 0.0;
      if (bad) atomicOr(flag, 1);
    }
  }
}

// Finite primitives with positive rho0, u_g and Ebar in every cell of a
// ghost-inclusive single-grid array [12][ncell].
__global__ void k_validate_cells(long long ncell, const double* __restrict__ P, int* flag) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < 12 * ncell;
       id += (long long)gridDim.x * blockDim.x) {
    const double v = P[id];
    const long long q = id / ncell;
    if (!isfinite(v) || ((q == hr::RHO || q == hr::UU || q == hr::ER) && !(v > 0.0))) atomicOr(flag, 1);
  }
}

__global__ void k_set_dt(double* dt, int nbox, double v) {
  for (int i = threadIdx.x; i < nbox; i += blockDim.x) dt[i] = v;
}

// Physics parameters shared by the grids of a context.
int fill_physics(const harmrad_params* p, DevParams& d) {
  memset(&d, 0, sizeof(d));
  for (int e = 0; e < 3; ++e) {
    if (p->n[e] < 1) return HARMRAD_E_ARG;
    d.act[e] = p->n[e] > 1 ? 1 : 0;
  }
  if (p->metric != 0 && p->metric != 1) return HARMRAD_E_ARG;
  d.metric = p->metric;
  d.a = p->a_spin;
  d.R0 = p->R0;
  d.h = p->hslope;
  if (p->metric == 1 && (fabs(p->a_spin) >= 1.0 || p->hslope <= 0.0 || p->hslope > 1.0)) return HARMRAD_E_ARG;
  if (!(p->gam > 1.0) || !(p->a_rad >= 0.0) || !(p->courant > 0.0)) return HARMRAD_E_ARG;
  d.gam = p->gam;
  d.a_rad = p->a_rad;
  d.courant = p->courant;
  if (p->opacity < 0 || p->opacity > 2) return HARMRAD_E_ARG;
  d.opacity = p->opacity;
  d.kabs0 = p->kappa_abs0;
  d.kes0 = p->kappa_es0;
  d.kscale = p->kappa_scale;
  d.Tmin = p->T_kappa_min;
  if (p->recon != 0 && p->recon != 1) return HARMRAD_E_ARG;
  if (p->flux != 0 && p->flux != 1) return HARMRAD_E_ARG;
  d.recon = p->recon;
  d.flux = p->flux;
  if (!(p->gamma_rad_max > 1.0) || !(p->gamma_gas_max > 1.0)) return HARMRAD_E_ARG;
  d.grad_max = p->gamma_rad_max;
  d.ggas_max = p->gamma_gas_max;
  // y_max of Eq. gammarvsy at gamma_rad_max: with s = sqrt(4-3y), 4 G (s-1) = s + 2
  double G2 = p->gamma_rad_max * p->gamma_rad_max;
  double s = (4.0 * G2 + 2.0) / (4.0 * G2 - 1.0);
  d.ymax_rad = (4.0 - s * s) / 3.0;
  d.rf0 = p->floor_rho0;
  d.rfp = p->floor_rho_pow;
  d.uf0 = p->floor_u0;
  d.ufp = p->floor_u_pow;
  if (!(p->bsq_rho_max > 0.0) || !(p->bsq_u_max > 0.0) || !(p->u_rho_max > 0.0)) return HARMRAD_E_ARG;
  d.bsq_rho_max = p->bsq_rho_max;
  d.bsq_u_max = p->bsq_u_max;
  d.u_rho_max = p->u_rho_max;
  if (p->newton_max < 1 || p->newton_max > 60) return HARMRAD_E_ARG;
  d.newton_max = p->newton_max;
  d.newton_tol = p->newton_tol;
  if (p->precision != 0 && p->precision != 1) return HARMRAD_E_ARG;
  d.precision = p->precision;
  // the entropy equation needs the RK3 stages (the IMEX sources cover the
  // energy-momentum rows only)
  if (p->implicit_eq != 0 && p->implicit_eq != 1) return HARMRAD_E_ARG;
  if (p->implicit_eq == 1 && p->integrator != 0) return HARMRAD_E_ARG;
  d.implicit_eq = p->implicit_eq;
  if (p->integrator < 0 || p->integrator > 3) return HARMRAD_E_ARG;
  d.integrator = p->integrator;
  if (p->emf != 0 && p->emf != 1) return HARMRAD_E_ARG;
  d.emf = p->emf;
  d.gm1f = (float)(d.gam - 1.0);
  d.ymaxf = (float)d.ymax_rad;
  d.Tminf = (float)d.Tmin;
  d.kabs0f = (float)d.kabs0;
  d.kes0f = (float)d.kes0;
  d.aradf = (float)d.a_rad;
  return HARMRAD_OK;
}

// Geometry of one grid (offsets left at zero).
int fill_geometry(const harmrad_params* p, BoxGeo& b) {
  memset(&b, 0, sizeof(b));
  long long ntot = 1, nact = 1;
  for (int e = 0; e < 3; ++e) {
    if (p->n[e] < 1) return HARMRAD_E_ARG;
    if (!(p->dx[e] > 0.0)) return HARMRAD_E_ARG;
    b.n[e] = p->n[e];
    b.ng[e] = p->n[e] > 1 ? 4 : 0;
    if (p->n[e] > 1 && p->n[e] < 4) return HARMRAD_E_ARG;  // ghosts need 4 active zones
    b.N[e] = b.n[e] + 2 * b.ng[e];
    ntot *= b.N[e];
    nact *= b.n[e];
    b.x0[e] = p->x0[e];
    b.dx[e] = p->dx[e];
  }
  b.ntot = ntot;
  b.nact = nact;
  b.goff = -1;
  b.str[0] = 1;
  b.str[1] = b.N[0];
  b.str[2] = (long long)b.N[0] * b.N[1];
  for (int s = 0; s < 6; ++s) {
    int bc = p->bc[s];
    if (bc < 0 || bc > 4) return HARMRAD_E_ARG;
    if (bc == 2 && (s / 2 != 1 || p->metric != 1)) return HARMRAD_E_ARG;
    b.bc[s] = bc;
  }
  if ((p->bc[2] == 2 || p->bc[3] == 2) && p->n[2] > 1 && (p->n[2] % 2)) return HARMRAD_E_ARG;
  return HARMRAD_OK;
}

// The grids of a batch share every parameter except sizes, coordinates and
// boundary conditions, and have the same active directions.
bool same_physics(const harmrad_params& a, const harmrad_params& b) {
  for (int e = 0; e < 3; ++e)
    if ((a.n[e] > 1) != (b.n[e] > 1)) return false;
  return a.metric == b.metric && a.a_spin == b.a_spin && a.R0 == b.R0 && a.hslope == b.hslope &&
         a.gam == b.gam && a.a_rad == b.a_rad && a.courant == b.courant && a.opacity == b.opacity &&
         a.kappa_abs0 == b.kappa_abs0 && a.kappa_es0 == b.kappa_es0 && a.kappa_scale == b.kappa_scale &&
         a.T_kappa_min == b.T_kappa_min && a.recon == b.recon && a.flux == b.flux &&
         a.gamma_rad_max == b.gamma_rad_max && a.gamma_gas_max == b.gamma_gas_max &&
         a.floor_rho0 == b.floor_rho0 && a.floor_rho_pow == b.floor_rho_pow && a.floor_u0 == b.floor_u0 &&
         a.floor_u_pow == b.floor_u_pow && a.bsq_rho_max == b.bsq_rho_max && a.bsq_u_max == b.bsq_u_max &&
         a.u_rho_max == b.u_rho_max && a.newton_max == b.newton_max && a.newton_tol == b.newton_tol &&
         a.precision == b.precision && a.integrator == b.integrator;
}

int run_faces(harmrad_ctx* c, bool fresh) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::faces(c, fresh) : hr::Run<hr::MINK>::faces(c, fresh);
}
int run_cfl(harmrad_ctx* c) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::cfl(c) : hr::Run<hr::MINK>::cfl(c);
}
int run_solve(harmrad_ctx* c, int s, const hr::ImexStage& im) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::solve(c, s, im) : hr::Run<hr::MINK>::solve(c, s, im);
}

// Sub-steps of a time integrator (Sec. 4.1): RK3 and IMEX2 have 3, IMEX2B 4,
// IMEX3 5 (its 4 implicit stages and the final combination).
int n_substeps(int integrator) { return integrator == 2 ? 4 : (integrator == 3 ? 5 : 3); }

// Sub-step k of an IMEX scheme as printed in Sec. 4.1 (Eqs. IMEX2, IMEX2B,
// IMEX3), one row {an, ap, d, c0, c1, c2, c3, g} per stage:
// U* = an U^n + ap U(P_prev) + d dt F(P_prev) + dt sum_j c_j M^j, solved with
// the implicit step g dt.
hr::ImexStage imex_stage(int integrator, int k) {
  hr::ImexStage s{};
  if (integrator == 0) return s;
  double row[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (integrator == 1) {
    const double y = 1.0 - 1.0 / sqrt(2.0);  // gamma
    const double t[3][8] = {{1, 0, 0, 0, 0, 0, 0, y},
                            {(3 * y - 1) / y, (1 - 2 * y) / y, 1, 0, 0, 0, 0, y},
                            {0.5, 0.5, 0.5, y, (1 - y) / 2, 0, 0, 0}};
    memcpy(row, t[k], sizeof(row));
  } else if (integrator == 2) {
    const double t[4][8] = {{1, 0, 0, 0, 0, 0, 0, 0.25},
                            {1, 0, 0.5, 0, 0, 0, 0, 0.25},
                            {0, 1, 0.5, 1.0 / 3, 1.0 / 12, 0, 0, 1.0 / 3},
                            {1.0 / 3, 2.0 / 3, 1.0 / 3, 1.0 / 9, 1.0 / 9, 1.0 / 9, 0, 0}};
    memcpy(row, t[k], sizeof(row));
  } else {
    const double a = 0.24169426078821, b = 0.06042356519705, e = 0.12915286960590;  // alpha, beta, eta
    const double t[5][8] = {
        {1, 0, 0, 0, 0, 0, 0, a},
        // [2U^n - U^0] as [U^n - alpha dt M^0]: the same by the first stage,
        // without subtracting the floors' additions to U^0
        {1, 0, 0, -a, 0, 0, 0, a},
        {1, 0, 1, 0, 1 - a, 0, 0, a},
        {0.75, 0.25, 0.25, b, (-1 + a + 4 * e) / 4, (2 - 5 * a - 4 * (b + e)) / 4, 0, a},
        {1.0 / 3, 2.0 / 3, 2.0 / 3, -2 * b / 3, (1 - 4 * e) / 6, (-1 + 4 * a + 4 * (b + e)) / 6, 4 * (1 - a) / 6, 0}};
    memcpy(row, t[k], sizeof(row));
  }
  s.an = row[0];
  s.ap = row[1];
  s.d = row[2];
  for (int j = 0; j < 4; ++j) s.c[j] = row[3 + j];
  s.g = row[7];
  s.on = 1;
  return s;
}

// Enqueue one full step.  with_cfl: the time step comes from the CFL pass of
// the current state, whose fluxes are then those of the first sub-step.
int enqueue_step(harmrad_ctx* c, bool with_cfl) {
  cudaStream_t st = c->stream;
  int nk = 0, r;
  if (c->adj)  // the adjoint recomputes the step from its input
    HR_CHECK(cudaMemcpyAsync(c->adj_Pn, c->P, 12 * (size_t)c->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                             st));
  HR_CHECK(cudaMemsetAsync(c->status, 0, c->nact, st));
  HR_CHECK(cudaMemsetAsync(c->iters, 0, c->nact * sizeof(int), st));
  HR_CHECK(cudaMemsetAsync(c->stats, 0, 8 * sizeof(unsigned long long), st));
  hr::mark(c, HARMRAD_K_OTHER);
  if (with_cfl) {
    if ((r = run_cfl(c)) < 0) return r;
    nk += r;
  }
  bool first = true;  // the first sub-step with fluxes restarts the flattener's maximum
  for (int s = 0; s < n_substeps(c->dp.integrator); ++s) {
    const hr::ImexStage im = imex_stage(c->dp.integrator, s);
    c->dp.sig_salt = s + 1;  // the branch signature tells the sub-steps apart
    if (!im.on || im.d != 0.0) {
      if (!(s == 0 && with_cfl)) {
        if ((r = run_faces(c, first)) < 0) return r;
        nk += r;
      }
      first = false;
    }
    if ((r = run_solve(c, s, im)) < 0) return r;
    nk += r;
  }
  c->dp.sig_salt = 0;
  return nk;
}

int launch_step(harmrad_ctx* c, bool with_cfl) {
  int gi = with_cfl ? 1 : 0;
  if (!c->use_graph) {
    int r = enqueue_step(c, with_cfl);
    if (r < 0) return r;
    c->launches_per_step = r;
    return HARMRAD_OK;
  }
  if (!c->graph[gi]) {
    cudaGraph_t g;
    HR_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int r = enqueue_step(c, with_cfl);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (r < 0) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return r;
    }
    HR_CHECK(e);
    cudaError_t ei = cudaGraphInstantiate(&c->graph[gi], g, 0);
    cudaGraphDestroy(g);
    HR_CHECK(ei);
    c->launches_per_step = r;
  }
  HR_CHECK(cudaGraphLaunch(c->graph[gi], c->stream));
  return HARMRAD_OK;
}

harmrad_tuning default_tuning() {
  harmrad_tuning t;
  memset(&t, 0, sizeof(t));
  t.face_block = 128;
  t.face_blocks_per_sm = 16;
  t.update_block = 128;
  t.update_blocks_per_sm = 16;
  t.edge_block = 256;
  t.edge_blocks_per_sm = 16;
  t.newton_split = 0;
  return t;
}

bool tuning_ok(const harmrad_tuning& t) {
  auto ok = [](int b, int cap, int bmax) { return b >= 32 && b <= bmax && b % 32 == 0 && cap >= 1 && cap <= 64; };
  return ok(t.face_block, t.face_blocks_per_sm, 128) && ok(t.update_block, t.update_blocks_per_sm, 128) &&
         ok(t.edge_block, t.edge_blocks_per_sm, 256) && t.newton_split >= 0 && t.newton_split <= 60;
}

void drop_graphs(harmrad_ctx* c) {
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) {
      cudaGraphExecDestroy(c->graph[g]);
      c->graph[g] = nullptr;
    }
}

void free_adjoint(harmrad_ctx* c) {
  if (c->adj) {
    hr::AdjBufs& a = *c->adj;
    void* ptrs[] = {a.Pst, a.chi, a.Ust, a.meth, a.Psol, a.gP, a.gN, a.gUn, a.gU, a.gX, a.gF[0], a.gF[1], a.gF[2],
                    a.gE, a.gchi, a.carry, a.gaux, a.gemf, a.gk, a.Sst, a.gS, a.gSn, a.gXS, a.gFS[0],
                    a.gFS[1], a.gFS[2]};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    delete c->adj;
    c->adj = nullptr;
  }
  if (c->adj_Pn) cudaFree(c->adj_Pn);
  c->adj_Pn = nullptr;
}

void free_all(harmrad_ctx* c) {
  free_adjoint(c);
  void* ptrs[] = {c->P, c->K, c->geotab, c->Un, c->F[0], c->F[1], c->F[2], c->spd[0], c->spd[1], c->spd[2],
                  c->aux, c->flat[0], c->flat[1], c->flat[2], c->emf, c->edges, c->slope, c->dt, c->status,
                  c->iters, c->failed, c->qcount, c->czone, c->cbox, c->cdata, c->qzone, c->qbox, c->qdata, c->fzone, c->fbox,
                  c->ftmp, c->stats, c->dtmin, c->stage_buf, c->flag, c->dboxes, c->imex_ust, c->imex_psol,
                  c->imex_M, c->sig, c->Sn, c->FS[0], c->FS[1], c->FS[2], c->Bf[0], c->Bf[1], c->Bf[2],
                  c->Bfn[0], c->Bfn[1], c->Bfn[2], c->gsp[0], c->gsp[1], c->gsp[2], c->vel, c->emf3[0],
                  c->emf3[1], c->emf3[2]};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (c->host_dt) cudaFreeHost(c->host_dt);
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
  for (int e = 0; e < 512; ++e)
    if (c->ev[e]) cudaEventDestroy(c->ev[e]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  free(c->boxes);
}

template <typename T>
int dalloc(T** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return HARMRAD_E_OOM;
  }
  return HARMRAD_OK;
}

int create(const harmrad_params* p, int count, void* stream, harmrad_ctx** out) {
  if (!p || !out || count < 1) return HARMRAD_E_ARG;
  *out = nullptr;
  DevParams dp;
  int rc = fill_physics(&p[0], dp);
  if (rc) return rc;
  std::vector<BoxGeo> boxes(count);
  long long coff = 0, aoff = 0, maxc = 0, maxa = 0, goff = 0;
  for (int b = 0; b < count; ++b) {
    if (b > 0 && !same_physics(p[0], p[b])) return HARMRAD_E_ARG;
    rc = fill_geometry(&p[b], boxes[b]);
    if (rc) return rc;
    boxes[b].coff = coff;
    boxes[b].aoff = aoff;
    if (dp.metric == 1) {
      boxes[b].goff = goff;
      goff += hr::geotab_size(boxes[b]);
    }
    coff += boxes[b].ntot;
    aoff += boxes[b].nact;
    maxc = boxes[b].ntot > maxc ? boxes[b].ntot : maxc;
    maxa = boxes[b].nact > maxa ? boxes[b].nact : maxa;
  }
  harmrad_ctx* c = (harmrad_ctx*)calloc(1, sizeof(harmrad_ctx));
  if (!c) return HARMRAD_E_OOM;
  c->prm = p[0];
  c->dp = dp;
  c->nbox = count;
  c->boxes = (BoxGeo*)malloc(sizeof(BoxGeo) * count);
  if (!c->boxes) {
    free(c);
    return HARMRAD_E_OOM;
  }
  memcpy(c->boxes, boxes.data(), sizeof(BoxGeo) * count);
  c->ncell = coff;
  c->nact = aoff;
  c->maxcell = maxc;
  c->maxact = maxa;
  c->real_size = p[0].precision == HARMRAD_PREC_SPLIT ? 4 : 8;
  c->use_graph = getenv("HARMRAD_NO_GRAPH") == nullptr;
  c->tune = default_tuning();
  if (count > 1) c->tune.newton_split = 3;  // batches: heavy-tailed Newton counts expected
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    free(c->boxes);
    free(c);
    return HARMRAD_E_CUDA;
  }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      cudaGetLastError();
      free(c->boxes);
      free(c);
      return HARMRAD_E_CUDA;
    }
    c->own_stream = true;
  }
  const size_t nt = c->ncell, na = c->nact, rs = c->real_size;
  const size_t nk = dp.opacity == 2 ? nt : 1;
  rc = HARMRAD_OK;
  rc = rc ? rc : dalloc(&c->dboxes, sizeof(BoxGeo) * count);
  rc = rc ? rc : dalloc(&c->P, 12 * nt * sizeof(double));
  rc = rc ? rc : dalloc(&c->K, nk * sizeof(double));
  if (goff > 0) rc = rc ? rc : dalloc(&c->geotab, goff * sizeof(double));
  rc = rc ? rc : dalloc(&c->Un, 12 * na * sizeof(double));
  if (dp.integrator == 0) rc = rc ? rc : dalloc(&c->Sn, na * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    size_t fn = dp.act[d] ? nt : 0;
    rc = rc ? rc : dalloc(&c->F[d], 12 * fn * rs);
    if (dp.integrator == 0 && fn) rc = rc ? rc : dalloc(&c->FS[d], fn * rs);
    rc = rc ? rc : dalloc(&c->spd[d], fn * rs);
    rc = rc ? rc : dalloc(&c->flat[d], 2 * fn * rs);
  }
  rc = rc ? rc : dalloc(&c->aux, 10 * nt * rs);
  rc = rc ? rc : dalloc(&c->emf, nt * rs);
  if (dp.emf == 1) {  // staggered field
    for (int d = 0; d < 3; ++d) {
      rc = rc ? rc : dalloc(&c->Bf[d], nt * sizeof(double));
      rc = rc ? rc : dalloc(&c->Bfn[d], nt * sizeof(double));
      rc = rc ? rc : dalloc(&c->gsp[d], 2 * nt * rs);
      rc = rc ? rc : dalloc(&c->emf3[d], nt * rs);
    }
    rc = rc ? rc : dalloc(&c->vel, 3 * nt * rs);
  }
  rc = rc ? rc : dalloc(&c->edges, 24 * nt * rs);
  rc = rc ? rc : dalloc(&c->slope, 12 * nt * rs);
  rc = rc ? rc : dalloc(&c->dt, count * sizeof(double));
  rc = rc ? rc : dalloc(&c->status, na);
  rc = rc ? rc : dalloc(&c->iters, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->failed, na);
  rc = rc ? rc : dalloc(&c->qcount, 4 * sizeof(int));
  rc = rc ? rc : dalloc(&c->czone, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->cbox, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->cdata, na * hr::CSTRIDE * sizeof(double));
  rc = rc ? rc : dalloc(&c->qzone, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->qbox, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->qdata, na * hr::QSTRIDE * sizeof(double));
  rc = rc ? rc : dalloc(&c->fzone, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->fbox, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->ftmp, na * 12 * sizeof(double));
  rc = rc ? rc : dalloc(&c->stats, 8 * sizeof(unsigned long long));
  rc = rc ? rc : dalloc(&c->dtmin, count * sizeof(unsigned long long));
  rc = rc ? rc : dalloc(&c->stage_buf, 12 * na * sizeof(double));
  if (dp.integrator != 0) {  // IMEX: U*, the implicit solutions and the stages' sources
    rc = rc ? rc : dalloc(&c->imex_ust, 12 * na * sizeof(double));
    rc = rc ? rc : dalloc(&c->imex_psol, 12 * na * sizeof(double));
    rc = rc ? rc : dalloc(&c->imex_M, 16 * na * sizeof(double));
  }
  rc = rc ? rc : dalloc(&c->flag, sizeof(int));
  if (!rc && cudaMallocHost((void**)&c->host_dt, count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = HARMRAD_E_OOM;
  }
  if (!rc) {
    // the grid table, and zeros in everything a kernel may read before writing
    if (cudaMemcpyAsync(c->dboxes, c->boxes, sizeof(BoxGeo) * count, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->P, 0, 12 * nt * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->K, 0, nk * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->stats, 0, 8 * sizeof(unsigned long long), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->status, 0, na, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->iters, 0, na * sizeof(int), c->stream) != cudaSuccess)
      rc = HARMRAD_E_CUDA;
    for (int d = 0; d < 3 && !rc; ++d) {
      size_t fn = dp.act[d] ? nt : 0;
      if (fn && c->FS[d] && cudaMemsetAsync(c->FS[d], 0, fn * rs, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
      if (fn && (cudaMemsetAsync(c->F[d], 0, 12 * fn * rs, c->stream) != cudaSuccess ||
                 cudaMemsetAsync(c->spd[d], 0, fn * rs, c->stream) != cudaSuccess ||
                 cudaMemsetAsync(c->flat[d], 0, 2 * fn * rs, c->stream) != cudaSuccess))
        rc = HARMRAD_E_CUDA;
    }
    if (!rc && c->geotab) {
      hr::k_geo_init<<<hr::grid_for(goff / 16, c->sms, 256), 256, 0, c->stream>>>(c->dp, c->dboxes, count,
                                                                                 c->geotab);
      if (cudaGetLastError() != cudaSuccess) rc = HARMRAD_E_CUDA;
    }
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  }
  if (rc) {
    free_all(c);
    free(c);
    return rc;
  }
  *out = c;
  return HARMRAD_OK;
}

int upload_planes(harmrad_ctx* c, int nv, const double* src_in, int on_device, double* dst) {
  size_t bytes = nv * (size_t)c->nact * sizeof(double);
  const double* src = src_in;
  if (!on_device) {
    HR_CHECK(cudaMemcpyAsync(c->stage_buf, src_in, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->stage_buf;
  }
  HR_CHECK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  int g = hr::grid_for(nv * c->maxact, c->sms, 256);
  k_validate<<<g, 256, 0, c->stream>>>(c->dboxes, c->nbox, nv, src, c->flag);
  k_unpack<<<g, 256, 0, c->stream>>>(c->dboxes, c->nbox, nv, src, dst);
  HR_CHECK(cudaGetLastError());
  int flag = 0;
  HR_CHECK(cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return flag ? HARMRAD_E_NAN_INPUT : HARMRAD_OK;
}

}  // namespace

// Parameter validation shared with the entry points in other translation units.
int harmrad_fill_params_internal(const harmrad_params* p, DevParams& d) { return fill_physics(p, d); }
int harmrad_fill_geometry_internal(const harmrad_params* p, BoxGeo& b) { return fill_geometry(p, b); }

extern "C" {

int harmrad_init(const harmrad_params* p, void* stream, harmrad_ctx** out) {
  return create(p, 1, stream, out);
}

int harmrad_init_batch(const harmrad_params* p, int count, void* stream, harmrad_ctx** out) {
  return create(p, count, stream, out);
}

void harmrad_destroy(harmrad_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  free(c);
}

// Staggered field: the faces from the cell-centred B just set (or, with
// from_centres false, the ghost faces and centres from the faces just set).
static int init_faces(harmrad_ctx* c, bool from_centres) {
  if (c->dp.emf != 1) return HARMRAD_OK;
  int r = c->dp.metric == 1 ? hr::Run<hr::KS>::init_faces(c, from_centres)
                            : hr::Run<hr::MINK>::init_faces(c, from_centres);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_set_prims(harmrad_ctx* c, const double* P, int on_device) {
  if (!c || !P) return HARMRAD_E_ARG;
  int rc = upload_planes(c, 12, P, on_device, c->P);
  if (rc) return rc;
  if ((rc = init_faces(c, true))) return rc;
  c->has_prims = true;
  return HARMRAD_OK;
}

int harmrad_set_face_fields(harmrad_ctx* c, const double* Bf, int on_device) {
  if (!c || !Bf || c->dp.emf != 1 || c->nbox != 1) return HARMRAD_E_ARG;
  const hr::BoxGeo& b = c->boxes[0];
  size_t n = 0;
  for (int d = 0; d < 3; ++d) {
    size_t m = 1;
    for (int e = 0; e < 3; ++e) m *= b.n[e] + ((e == d && b.n[d] > 1) ? 1 : 0);
    n += m;
  }
  // host data stage through the [12][nact] staging buffer: the face count
  // of a grid, at most 3 (n1+1)(n2+1)(n3+1) <= 12 n1 n2 n3 when every n >= 1
  double* src = (double*)Bf;
  if (!on_device) {
    HR_CHECK(cudaMemcpyAsync(c->stage_buf, Bf, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = c->stage_buf;
  }
  hr::FaceSet fs;
  for (int d = 0; d < 3; ++d) fs.f[d] = c->Bf[d];
  hr::k_face_pack<<<hr::grid_for((long long)n, c->sms, 256), 256, 0, c->stream>>>(c->dboxes, src, fs, true);
  HR_CHECK(cudaGetLastError());
  return init_faces(c, false);
}

int harmrad_get_face_fields(harmrad_ctx* c, double* Bf, int on_device) {
  if (!c || !Bf || c->dp.emf != 1 || c->nbox != 1) return HARMRAD_E_ARG;
  const hr::BoxGeo& b = c->boxes[0];
  size_t n = 0;
  for (int d = 0; d < 3; ++d) {
    size_t m = 1;
    for (int e = 0; e < 3; ++e) m *= b.n[e] + ((e == d && b.n[d] > 1) ? 1 : 0);
    n += m;
  }
  double* dst = on_device ? Bf : c->stage_buf;
  hr::FaceSet fs;
  for (int d = 0; d < 3; ++d) fs.f[d] = c->Bf[d];
  hr::k_face_pack<<<hr::grid_for((long long)n, c->sms, 256), 256, 0, c->stream>>>(c->dboxes, dst, fs, false);
  HR_CHECK(cudaGetLastError());
  if (!on_device)
    HR_CHECK(cudaMemcpyAsync(Bf, c->stage_buf, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_set_prims_ghosts(harmrad_ctx* c, const double* P, int on_device) {
  if (!c || !P || c->nbox != 1) return HARMRAD_E_ARG;
  const size_t bytes = 12 * (size_t)c->ncell * sizeof(double);
  HR_CHECK(cudaMemcpyAsync(c->P, P, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->stream));
  HR_CHECK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  k_validate_cells<<<hr::grid_for(c->ncell, c->sms, 256), 256, 0, c->stream>>>(c->ncell, c->P, c->flag);
  HR_CHECK(cudaGetLastError());
  int flag = 0;
  HR_CHECK(cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  if (flag) return HARMRAD_E_NAN_INPUT;
  int rc = init_faces(c, true);
  if (rc) return rc;
  c->has_prims = true;
  return HARMRAD_OK;
}

int harmrad_set_opacity_field(harmrad_ctx* c, const double* kabs, int on_device) {
  if (!c || !kabs) return HARMRAD_E_ARG;
  if (c->dp.opacity != HARMRAD_OPAC_FIELD) return HARMRAD_E_ARG;
  return upload_planes(c, 1, kabs, on_device, c->K);
}

int harmrad_get_prims(harmrad_ctx* c, double* P, int on_device) {
  if (!c || !P) return HARMRAD_E_ARG;
  size_t bytes = 12 * (size_t)c->nact * sizeof(double);
  int g = hr::grid_for(12 * c->maxact, c->sms, 256);
  double* dst = on_device ? P : c->stage_buf;
  k_pack<<<g, 256, 0, c->stream>>>(c->dboxes, c->nbox, c->P, dst);
  HR_CHECK(cudaGetLastError());
  if (!on_device) {
    HR_CHECK(cudaMemcpyAsync(P, c->stage_buf, bytes, cudaMemcpyDeviceToHost, c->stream));
    HR_CHECK(cudaStreamSynchronize(c->stream));
  }
  return HARMRAD_OK;
}

int harmrad_cfl_dt(harmrad_ctx* c, double* dt) {
  if (!c || !dt) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  int r = run_cfl(c);
  if (r < 0) return r;
  HR_CHECK(cudaMemcpyAsync(c->host_dt, c->dt, c->nbox * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  double m = c->host_dt[0];
  for (int b = 1; b < c->nbox; ++b) m = c->host_dt[b] < m ? c->host_dt[b] : m;
  *dt = m;
  return HARMRAD_OK;
}

int harmrad_step(harmrad_ctx* c, double dt) {
  if (!c) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  bool with_cfl = !(dt > 0.0);
  if (!with_cfl) {
    // the value travels as a kernel argument: no host synchronisation
    k_set_dt<<<1, 128, 0, c->stream>>>(c->dt, c->nbox, dt);
    HR_CHECK(cudaGetLastError());
  }
  c->last_dt = dt;
  int r = launch_step(c, with_cfl);
  c->adj_ready = c->adj != nullptr && r == HARMRAD_OK;
  return r;
}

int harmrad_profile_step(harmrad_ctx* c, double dt, harmrad_kernel_times* out) {
  if (!c || !out) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  memset(out, 0, sizeof(*out));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  bool with_cfl = !(dt > 0.0);
  c->profiling = true;
  c->nev = 0;
  hr::mark(c, HARMRAD_K_OTHER);  // start marker
  int r = 0;
  if (!with_cfl) {
    k_set_dt<<<1, 128, 0, c->stream>>>(c->dt, c->nbox, dt);
    hr::mark(c, HARMRAD_K_OTHER);
  }
  r = enqueue_step(c, with_cfl);
  c->profiling = false;
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(c->stream));
  for (int e = 1; e < c->nev; ++e) {
    float ms = 0.0f;
    HR_CHECK(cudaEventElapsedTime(&ms, c->ev[e - 1], c->ev[e]));
    int t = c->ev_tag[e];
    out->ms[t] += ms;
    out->launches[t] += 1;
  }
  out->total_launches = r;
  return HARMRAD_OK;
}

int harmrad_step_host(harmrad_ctx* c, const double* P_in, double* P_out, double dt) {
  if (!c || !P_in || !P_out) return HARMRAD_E_ARG;
  int r = harmrad_set_prims(c, P_in, 0);
  if (r) return r;
  r = harmrad_step(c, dt);
  if (r) return r;
  return harmrad_get_prims(c, P_out, 0);
}

int harmrad_get_stats(harmrad_ctx* c, harmrad_stats* s) {
  if (!c || !s) return HARMRAD_E_ARG;
  unsigned long long h[8];
  HR_CHECK(cudaMemcpyAsync(h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaMemcpyAsync(c->host_dt, c->dt, c->nbox * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  double m = c->host_dt[0];
  for (int b = 1; b < c->nbox; ++b) m = c->host_dt[b] < m ? c->host_dt[b] : m;
  s->dt = m;
  s->pmhd_ok = (long long)h[hr::ST_PMHD];
  s->urad_ok = (long long)h[hr::ST_URAD];
  s->backup = (long long)h[hr::ST_BACKUP];
  s->zone_stages = (long long)h[hr::ST_SOLVES];
  s->newton_iters = (long long)h[hr::ST_ITERS];
  s->entropy_ok = (long long)h[hr::ST_ENTROPY];
  s->cold_ok = (long long)h[hr::ST_COLD];
  s->kernel_launches = c->launches_per_step;
  s->graph = c->use_graph ? 1 : 0;
  return s->backup > 0 ? HARMRAD_W_BACKUP_USED : HARMRAD_OK;
}

int harmrad_get_status(harmrad_ctx* c, unsigned char* st, int on_device) {
  if (!c || !st) return HARMRAD_E_ARG;
  HR_CHECK(cudaMemcpyAsync(st, c->status, c->nact,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_get_iters(harmrad_ctx* c, int* it, int on_device) {
  if (!c || !it) return HARMRAD_E_ARG;
  HR_CHECK(cudaMemcpyAsync(it, c->iters, c->nact * sizeof(int),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_compute_fluxes(harmrad_ctx* c, int dir, double* F_host) {
  if (!c || !F_host || dir < 1 || dir > 3) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  if (c->nbox != 1) return HARMRAD_E_ARG;
  const BoxGeo& b = c->boxes[0];
  int d = dir - 1;
  if (b.n[d] == 1) return HARMRAD_E_ARG;
  int r = run_faces(c, true);
  if (r < 0) return r;
  size_t rs = c->real_size;
  size_t bytes = 12 * (size_t)b.ntot * rs;
  char* hbuf = (char*)malloc(bytes);
  if (!hbuf) return HARMRAD_E_OOM;
  if (cudaMemcpyAsync(hbuf, c->F[d], bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    free(hbuf);
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  int m[3] = {b.n[0], b.n[1], b.n[2]};
  m[d] += 1;
  long long nf = (long long)m[0] * m[1] * m[2];
  for (int q = 0; q < 12; ++q)
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i) {
          long long t = hr::cell_index(b, i, j, k);
          long long o = (long long)q * nf + ((long long)k * m[1] + j) * m[0] + i;
          F_host[o] = rs == 8 ? ((double*)hbuf)[q * b.ntot + t] : (double)((float*)hbuf)[q * b.ntot + t];
        }
  free(hbuf);
  return HARMRAD_OK;
}

int harmrad_zone_physics(const harmrad_params* prm, int n, const double* x, const double* P, double* U,
                         double* SM, double* F, double* speeds, void* stream) {
  if (!prm || n < 0 || (n > 0 && (!x || !P))) return HARMRAD_E_ARG;
  DevParams dp;
  BoxGeo bg;
  int rc = fill_physics(prm, dp);
  if (!rc) rc = fill_geometry(prm, bg);
  if (rc) return rc;
  if (dp.opacity == HARMRAD_OPAC_FIELD) return HARMRAD_E_ARG;
  if (n == 0) return HARMRAD_OK;
  int dev, sms;
  HR_CHECK(cudaGetDevice(&dev));
  HR_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int r = dp.metric == 1 ? hr::Run<hr::KS>::zone_physics(dp, bg, n, x, P, U, SM, F, speeds, st, sms)
                         : hr::Run<hr::MINK>::zone_physics(dp, bg, n, x, P, U, SM, F, speeds, st, sms);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(st));
  return HARMRAD_OK;
}

static int zone_implicit_impl(const harmrad_params* prm, int n, const double* x, const double* Us,
                              const double* Ss, const double* Ps, const double* h, double* Pout, double* eT,
                              int* iters, unsigned char* method, void* stream) {
  if (!prm || n < 0 || (n > 0 && (!x || !Us || !Ps || !h || !Pout))) return HARMRAD_E_ARG;
  DevParams dp;
  BoxGeo bg;
  int rc = fill_physics(prm, dp);
  if (!rc) rc = fill_geometry(prm, bg);
  if (rc) return rc;
  if (dp.opacity == HARMRAD_OPAC_FIELD) return HARMRAD_E_ARG;
  if (n == 0) return HARMRAD_OK;
  int dev, sms;
  HR_CHECK(cudaGetDevice(&dev));
  HR_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int r = dp.metric == 1
              ? hr::Run<hr::KS>::zone_implicit(dp, bg, n, x, Us, Ss, Ps, h, Pout, eT, iters, method, st, sms)
              : hr::Run<hr::MINK>::zone_implicit(dp, bg, n, x, Us, Ss, Ps, h, Pout, eT, iters, method, st, sms);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(st));
  return HARMRAD_OK;
}

int harmrad_zone_implicit(const harmrad_params* prm, int n, const double* x, const double* Us,
                          const double* Ps, const double* h, double* Pout, double* eT, int* iters,
                          unsigned char* method, void* stream) {
  return zone_implicit_impl(prm, n, x, Us, nullptr, Ps, h, Pout, eT, iters, method, stream);
}

int harmrad_zone_method(const harmrad_params* prm, int n, const double* x, const double* Us, const double* Sstar,
                        const double* Ps, const double* h, int method, double* Pout, double* eT, int* iters,
                        void* stream) {
  if (!prm || n < 0 || method < 0 || method > 8 || (method >= 6 && !Sstar) ||
      (n > 0 && (!x || !Us || !Ps || !h || !Pout || !eT || !iters)))
    return HARMRAD_E_ARG;
  DevParams dp;
  BoxGeo bg;
  int rc = fill_physics(prm, dp);
  if (!rc) rc = fill_geometry(prm, bg);
  if (rc) return rc;
  if (dp.opacity == HARMRAD_OPAC_FIELD) return HARMRAD_E_ARG;
  if (n == 0) return HARMRAD_OK;
  int dev, sms;
  HR_CHECK(cudaGetDevice(&dev));
  HR_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int r = dp.metric == 1
              ? hr::Run<hr::KS>::zone_method(dp, bg, n, x, Us, Sstar, Ps, h, method, Pout, eT, iters, st, sms)
              : hr::Run<hr::MINK>::zone_method(dp, bg, n, x, Us, Sstar, Ps, h, method, Pout, eT, iters, st, sms);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(st));
  return HARMRAD_OK;
}

int harmrad_zone_implicit_full(const harmrad_params* prm, int n, const double* x, const double* Us,
                               const double* Sstar, const double* Ps, const double* h, double* Pout,
                               double* eT, int* iters, unsigned char* method, void* stream) {
  return zone_implicit_impl(prm, n, x, Us, Sstar, Ps, h, Pout, eT, iters, method, stream);
}

int harmrad_adjoint_enable(harmrad_ctx* c, int on) {
  if (!c) return HARMRAD_E_ARG;
  HR_CHECK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  c->adj_ready = false;
  if (!on) {
    free_adjoint(c);
    return HARMRAD_OK;
  }
  if (c->nbox != 1 || c->real_size != 8 || c->dp.integrator != 0 || c->dp.implicit_eq != 0 || c->dp.emf != 0)
    return HARMRAD_E_ARG;
  for (int f = 0; f < 6; ++f)
    if (c->boxes[0].bc[f] == HARMRAD_BC_FIXED) return HARMRAD_E_ARG;
  if (c->adj) return HARMRAD_OK;
  c->adj = new hr::AdjBufs();
  memset(c->adj, 0, sizeof(hr::AdjBufs));
  hr::AdjBufs& a = *c->adj;
  const size_t nt = c->ncell, na = c->nact, D = sizeof(double);
  int rc = HARMRAD_OK;
  rc = rc ? rc : dalloc(&c->adj_Pn, 12 * nt * D);
  rc = rc ? rc : dalloc(&a.Pst, 4 * 12 * nt * D);
  rc = rc ? rc : dalloc(&a.chi, 3 * 3 * 2 * nt * D);
  rc = rc ? rc : dalloc(&a.Ust, 3 * 12 * na * D);
  rc = rc ? rc : dalloc(&a.meth, 3 * na);
  rc = rc ? rc : dalloc(&a.Psol, 3 * 12 * na * D);
  rc = rc ? rc : dalloc(&a.gP, 12 * nt * D);
  rc = rc ? rc : dalloc(&a.gN, 12 * na * D);
  rc = rc ? rc : dalloc(&a.gUn, 12 * na * D);
  rc = rc ? rc : dalloc(&a.gU, 12 * na * D);
  rc = rc ? rc : dalloc(&a.gX, 12 * na * D);
  for (int d = 0; d < 3; ++d) rc = rc ? rc : dalloc(&a.gF[d], 12 * nt * D);
  rc = rc ? rc : dalloc(&a.gE, 24 * nt * D);
  rc = rc ? rc : dalloc(&a.gchi, 2 * nt * D);
  rc = rc ? rc : dalloc(&a.carry, 6 * nt * D);
  rc = rc ? rc : dalloc(&a.gaux, 3 * nt * D);
  rc = rc ? rc : dalloc(&a.gemf, nt * D);
  rc = rc ? rc : dalloc(&a.gk, D);
  rc = rc ? rc : dalloc(&a.Sst, 3 * na * D);
  rc = rc ? rc : dalloc(&a.gS, na * D);
  rc = rc ? rc : dalloc(&a.gSn, na * D);
  rc = rc ? rc : dalloc(&a.gXS, na * D);
  for (int d = 0; d < 3; ++d) rc = rc ? rc : dalloc(&a.gFS[d], nt * D);
  if (!rc && cudaMemsetAsync(a.chi, 0, 3 * 3 * 2 * nt * D, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (!rc && cudaMemsetAsync(a.gF[0], 0, 12 * nt * D, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (!rc && cudaMemsetAsync(a.gF[1], 0, 12 * nt * D, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (!rc && cudaMemsetAsync(a.gF[2], 0, 12 * nt * D, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (rc) free_adjoint(c);
  return rc;
}

int harmrad_branch_signature(harmrad_ctx* c, int on) {
  if (!c) return HARMRAD_E_ARG;
  HR_CHECK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);  // the captured launches carry the signature pointer
  if (!on) {
    if (c->sig) cudaFree(c->sig);
    c->sig = nullptr;
    c->dp.sig = nullptr;
    return HARMRAD_OK;
  }
  if (!c->sig && dalloc(&c->sig, c->ncell * sizeof(unsigned long long)) != HARMRAD_OK) return HARMRAD_E_OOM;
  HR_CHECK(cudaMemsetAsync(c->sig, 0, c->ncell * sizeof(unsigned long long), c->stream));
  c->dp.sig = c->sig;
  return HARMRAD_OK;
}

int harmrad_get_branch_signature(harmrad_ctx* c, unsigned long long* out, int on_device) {
  if (!c || !out) return HARMRAD_E_ARG;
  if (!c->sig) return HARMRAD_E_STATE;
  HR_CHECK(cudaMemcpyAsync(out, c->sig, c->ncell * sizeof(unsigned long long),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_adjoint_set_input(harmrad_ctx* c, const double* P, double dt, int on_device) {
  if (!c || !P || !(dt > 0.0)) return HARMRAD_E_ARG;
  if (!c->adj) return HARMRAD_E_STATE;
  int rc = harmrad_set_prims(c, P, on_device);
  if (rc) return rc;
  // what harmrad_step records for the adjoint: its input and its time step
  HR_CHECK(cudaMemcpyAsync(c->adj_Pn, c->P, 12 * (size_t)c->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                           c->stream));
  k_set_dt<<<1, 128, 0, c->stream>>>(c->dt, c->nbox, dt);
  HR_CHECK(cudaGetLastError());
  c->last_dt = dt;
  c->adj_ready = true;
  return HARMRAD_OK;
}

int harmrad_step_adjoint(harmrad_ctx* c, const double* gP_out, double* gP_in, double* g_kappa, int on_device) {
  if (!c || !gP_out || !gP_in) return HARMRAD_E_ARG;
  if (!c->adj || !c->adj_ready) return HARMRAD_E_STATE;
  const size_t bytes = 12 * (size_t)c->nact * sizeof(double);
  const double* gin = gP_out;
  double* gout = gP_in;
  if (!on_device) {  // stage through the cotangent buffers of the workspace
    HR_CHECK(cudaMemcpyAsync(c->stage_buf, gP_out, bytes, cudaMemcpyHostToDevice, c->stream));
    gin = c->stage_buf;
    gout = c->stage_buf;
  }
  int r = c->dp.metric == 1 ? hr::Run<hr::KS>::adjoint(c, gin, gout, nullptr)
                            : hr::Run<hr::MINK>::adjoint(c, gin, gout, nullptr);
  if (r < 0) return r;
  double gk = 0.0;
  HR_CHECK(cudaMemcpyAsync(&gk, c->adj->gk, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (!on_device) HR_CHECK(cudaMemcpyAsync(gP_in, c->stage_buf, bytes, cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  if (g_kappa) *g_kappa = gk;
  return HARMRAD_OK;
}

int harmrad_get_tuning(harmrad_ctx* c, harmrad_tuning* out) {
  if (!c || !out) return HARMRAD_E_ARG;
  *out = c->tune;
  return HARMRAD_OK;
}

int harmrad_set_tuning(harmrad_ctx* c, const harmrad_tuning* t) {
  if (!c || !t || !tuning_ok(*t)) return HARMRAD_E_ARG;
  HR_CHECK(cudaStreamSynchronize(c->stream));
  c->tune = *t;
  drop_graphs(c);
  return HARMRAD_OK;
}

int harmrad_autotune(harmrad_ctx* c, int reps, harmrad_tuning* out) {
  if (!c) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  if (reps < 1) reps = 1;
  struct Shape {
    int block, cap, split;
  };
  // candidate i pairs the i-th shape of each class; the classes are timed
  // separately within the same step
  const Shape fc[] = {{128, 16, 0}, {64, 16, 0}, {128, 8, 0}, {128, 32, 0}, {64, 32, 0},
                      {128, 64, 0}, {128, 4, 0}, {128, 32, 0}, {64, 64, 0}};
  const Shape uc[] = {{128, 16, 0}, {64, 16, 3}, {128, 8, 5}, {128, 32, 0}, {64, 32, 3},
                      {128, 64, 3}, {64, 64, 0}, {128, 32, 3}, {128, 32, 5}};
  const Shape ec[] = {{256, 16, 0}, {128, 16, 0}, {256, 8, 0}, {256, 32, 0}, {128, 32, 0},
                      {256, 64, 0}, {128, 64, 0}, {256, 32, 0}, {128, 8, 0}};
  const int ncand = 9;
  const size_t bytes = 12 * (size_t)c->ncell * sizeof(double);
  double* save = nullptr;
  if (cudaMalloc((void**)&save, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_OOM;
  }
  const harmrad_tuning orig = c->tune;
  harmrad_tuning best = orig;
  best.face_ms = best.update_ms = best.edge_ms = HUGE_VAL;
  int rc = HARMRAD_OK;
  if (cudaMemcpyAsync(save, c->P, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) rc = HARMRAD_E_CUDA;
  for (int it = -1; it < reps * ncand && rc >= 0; ++it) {
    harmrad_tuning t = orig;
    if (it >= 0) {  // it = -1: one untimed step loads every kernel
      int i = it % ncand;
      t.face_block = fc[i].block;
      t.face_blocks_per_sm = fc[i].cap;
      t.update_block = uc[i].block;
      t.update_blocks_per_sm = uc[i].cap;
      t.newton_split = uc[i].split;
      t.edge_block = ec[i].block;
      t.edge_blocks_per_sm = ec[i].cap;
    }
    c->tune = t;
    harmrad_kernel_times kt;
    rc = harmrad_profile_step(c, 0.0, &kt);
    if (rc < 0) break;
    if (cudaMemcpyAsync(c->P, save, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
      rc = HARMRAD_E_CUDA;
      break;
    }
    if (it < 0) continue;
    if (kt.ms[HARMRAD_K_FACE] < best.face_ms) {
      best.face_ms = kt.ms[HARMRAD_K_FACE];
      best.face_block = t.face_block;
      best.face_blocks_per_sm = t.face_blocks_per_sm;
    }
    if (kt.ms[HARMRAD_K_UPDATE] < best.update_ms) {
      best.update_ms = kt.ms[HARMRAD_K_UPDATE];
      best.update_block = t.update_block;
      best.update_blocks_per_sm = t.update_blocks_per_sm;
      best.newton_split = t.newton_split;
    }
    if (kt.ms[HARMRAD_K_EDGE] < best.edge_ms) {
      best.edge_ms = kt.ms[HARMRAD_K_EDGE];
      best.edge_block = t.edge_block;
      best.edge_blocks_per_sm = t.edge_blocks_per_sm;
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess && rc >= 0) rc = HARMRAD_E_CUDA;
  cudaFree(save);
  if (rc < 0) {
    c->tune = orig;
    return rc;
  }
  c->tune = best;
  drop_graphs(c);
  if (out) *out = best;
  return HARMRAD_OK;
}

const char* harmrad_strerror(int code) {
  switch (code) {
    case HARMRAD_OK: return "ok";
    case HARMRAD_W_BACKUP_USED: return "warning: some zones used the neighbour-average back-up";
    case HARMRAD_E_ARG: return "invalid argument";
    case HARMRAD_E_CUDA: return "CUDA runtime error";
    case HARMRAD_E_OOM: return "out of device memory";
    case HARMRAD_E_NAN_INPUT: return "input not finite or out of range";
    case HARMRAD_E_STATE: return "call out of order (no primitives loaded)";
    default: return "unknown harmrad return code";
  }
}

}  // extern "C"
