// C ABI of the harmrad library: context management, data movement and the
// sequence of one full RK3 step (Sec. 4.1-4.2 of McKinney et al. 2014),
// replayed as a CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hr_ctx.h"

using hr::DevParams;

namespace {

#define HR_CHECK(x)                          \
  do {                                       \
    if ((x) != cudaSuccess) {                \
      cudaGetLastError();                    \
      return HARMRAD_E_CUDA;                 \
    }                                        \
  } while (0)

// active layout [12][n3][n2][n1] <-> ghost-inclusive layout
__global__ void k_unpack(DevParams p, const double* __restrict__ src, double* __restrict__ P) {
  long long total = (long long)hr::NPR * p.nact;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    long long q = id / p.nact, z = id % p.nact, r = z;
    int i = (int)(r % p.n[0]);
    r /= p.n[0];
    int j = (int)(r % p.n[1]);
    int k = (int)(r / p.n[1]);
    P[q * p.ntot + hr::cell_index(p, i, j, k)] = src[id];
  }
}

__global__ void k_pack(DevParams p, const double* __restrict__ P, double* __restrict__ dst) {
  long long total = (long long)hr::NPR * p.nact;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    long long q = id / p.nact, z = id % p.nact, r = z;
    int i = (int)(r % p.n[0]);
    r /= p.n[0];
    int j = (int)(r % p.n[1]);
    int k = (int)(r / p.n[1]);
    dst[id] = P[q * p.ntot + hr::cell_index(p, i, j, k)];
  }
}

// flag = 1 if any value is not finite or rho0, u_g, Ebar is not positive
__global__ void k_validate(DevParams p, const double* __restrict__ src, int* flag) {
  long long total = (long long)hr::NPR * p.nact;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    double v = src[id];
    long long q = id / p.nact;
    bool bad = !isfinite(v) || ((q == hr::RHO || q == hr::UU || q == hr::ER) && !(v > 0.0));
    if (bad) atomicOr(flag, 1);
  }
}

__global__ void k_set_dt(double* dt, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dt = v;
}

int fill_devparams(const harmrad_params* p, DevParams& d) {
  memset(&d, 0, sizeof(d));
  long long ntot = 1, nact = 1;
  for (int e = 0; e < 3; ++e) {
    if (p->n[e] < 1) return HARMRAD_E_ARG;
    if (!(p->dx[e] > 0.0)) return HARMRAD_E_ARG;
    d.n[e] = p->n[e];
    d.ng[e] = p->n[e] > 1 ? 4 : 0;
    if (p->n[e] > 1 && p->n[e] < 4) return HARMRAD_E_ARG;  // ghosts need 4 active zones
    d.N[e] = d.n[e] + 2 * d.ng[e];
    ntot *= d.N[e];
    nact *= d.n[e];
    d.x0[e] = p->x0[e];
    d.dx[e] = p->dx[e];
  }
  d.ntot = ntot;
  d.nact = nact;
  d.str[0] = 1;
  d.str[1] = d.N[0];
  d.str[2] = (long long)d.N[0] * d.N[1];
  if (p->metric != 0 && p->metric != 1) return HARMRAD_E_ARG;
  d.metric = p->metric;
  d.a = p->a_spin;
  d.R0 = p->R0;
  d.h = p->hslope;
  if (p->metric == 1 && (fabs(p->a_spin) >= 1.0 || p->hslope <= 0.0 || p->hslope > 1.0)) return HARMRAD_E_ARG;
  for (int s = 0; s < 6; ++s) {
    int bc = p->bc[s];
    if (bc < 0 || bc > 2) return HARMRAD_E_ARG;
    if (bc == 2 && (s / 2 != 1 || p->metric != 1)) return HARMRAD_E_ARG;
    d.bc[s] = bc;
  }
  if ((p->bc[2] == 2 || p->bc[3] == 2) && p->n[2] > 1 && (p->n[2] % 2)) return HARMRAD_E_ARG;
  if (!(p->gam > 1.0) || !(p->a_rad >= 0.0) || !(p->courant > 0.0)) return HARMRAD_E_ARG;
  d.gam = p->gam;
  d.a_rad = p->a_rad;
  d.courant = p->courant;
  if (p->opacity != 0 && p->opacity != 1) return HARMRAD_E_ARG;
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
  return HARMRAD_OK;
}

int run_faces(harmrad_ctx* c, bool fresh) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::faces(c, fresh) : hr::Run<hr::MINK>::faces(c, fresh);
}
int run_cfl(harmrad_ctx* c) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::cfl(c) : hr::Run<hr::MINK>::cfl(c);
}
int run_solve(harmrad_ctx* c, int s) {
  return c->dp.metric == 1 ? hr::Run<hr::KS>::solve(c, s) : hr::Run<hr::MINK>::solve(c, s);
}

// Enqueue one full step.  with_cfl: the time step comes from the CFL pass of
// the current state, whose fluxes are then those of the first sub-step.
int enqueue_step(harmrad_ctx* c, bool with_cfl) {
  const DevParams& p = c->dp;
  cudaStream_t st = c->stream;
  int nk = 0, r;
  HR_CHECK(cudaMemsetAsync(c->status, 0, p.nact, st));
  HR_CHECK(cudaMemsetAsync(c->iters, 0, p.nact * sizeof(int), st));
  HR_CHECK(cudaMemsetAsync(c->stats, 0, 8 * sizeof(unsigned long long), st));
  hr::mark(c, HARMRAD_K_OTHER);
  if (with_cfl) {
    if ((r = run_cfl(c)) < 0) return r;
    nk += r;
  }
  for (int s = 0; s < 3; ++s) {
    if (!(s == 0 && with_cfl)) {
      if ((r = run_faces(c, s == 0)) < 0) return r;
      nk += r;
    }
    if ((r = run_solve(c, s)) < 0) return r;
    nk += r;
  }
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

void free_all(harmrad_ctx* c) {
  void* ptrs[] = {c->P, c->Un, c->F[0], c->F[1], c->F[2], c->spd[0], c->spd[1], c->spd[2],
                  c->aux, c->flat[0], c->flat[1], c->flat[2], c->emf, c->edges, c->dt, c->status, c->iters,
                  c->failed, c->qcount, c->qzone, c->qdata, c->fzone, c->ftmp, c->stats, c->dtmin,
                  c->stage_buf, c->flag};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (c->host_dt) cudaFreeHost(c->host_dt);
  for (int g = 0; g < 2; ++g)
    if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
  for (int e = 0; e < 512; ++e)
    if (c->ev[e]) cudaEventDestroy(c->ev[e]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
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

}  // namespace

// Parameter validation shared with the entry points in other translation units.
int harmrad_fill_params_internal(const harmrad_params* p, DevParams& d) { return fill_devparams(p, d); }

extern "C" {

int harmrad_init(const harmrad_params* p, void* stream, harmrad_ctx** out) {
  if (!p || !out) return HARMRAD_E_ARG;
  *out = nullptr;
  DevParams dp;
  int rc = fill_devparams(p, dp);
  if (rc) return rc;
  harmrad_ctx* c = (harmrad_ctx*)calloc(1, sizeof(harmrad_ctx));
  if (!c) return HARMRAD_E_OOM;
  c->prm = *p;
  c->dp = dp;
  c->real_size = p->precision == HARMRAD_PREC_SPLIT ? 4 : 8;
  c->use_graph = getenv("HARMRAD_NO_GRAPH") == nullptr;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    free(c);
    return HARMRAD_E_CUDA;
  }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      cudaGetLastError();
      free(c);
      return HARMRAD_E_CUDA;
    }
    c->own_stream = true;
  }
  const size_t nt = dp.ntot, na = dp.nact, rs = c->real_size;
  rc = HARMRAD_OK;
  rc = rc ? rc : dalloc(&c->P, 12 * nt * sizeof(double));
  rc = rc ? rc : dalloc(&c->Un, 12 * na * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    size_t fn = dp.n[d] > 1 ? nt : 0;
    rc = rc ? rc : dalloc(&c->F[d], 12 * fn * rs);
    rc = rc ? rc : dalloc(&c->spd[d], fn * rs);
    rc = rc ? rc : dalloc(&c->flat[d], 2 * fn * rs);
  }
  rc = rc ? rc : dalloc(&c->aux, 10 * nt * rs);
  rc = rc ? rc : dalloc(&c->emf, nt * rs);
  rc = rc ? rc : dalloc(&c->edges, 24 * nt * rs);
  rc = rc ? rc : dalloc(&c->dt, sizeof(double));
  rc = rc ? rc : dalloc(&c->status, na);
  rc = rc ? rc : dalloc(&c->iters, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->failed, na);
  rc = rc ? rc : dalloc(&c->qcount, 2 * sizeof(int));
  rc = rc ? rc : dalloc(&c->qzone, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->qdata, na * hr::QSTRIDE * sizeof(double));
  rc = rc ? rc : dalloc(&c->fzone, na * sizeof(int));
  rc = rc ? rc : dalloc(&c->ftmp, na * 12 * sizeof(double));
  rc = rc ? rc : dalloc(&c->stats, 8 * sizeof(unsigned long long));
  rc = rc ? rc : dalloc(&c->dtmin, sizeof(unsigned long long));
  rc = rc ? rc : dalloc(&c->stage_buf, 12 * na * sizeof(double));
  rc = rc ? rc : dalloc(&c->flag, sizeof(int));
  if (!rc && cudaMallocHost((void**)&c->host_dt, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = HARMRAD_E_OOM;
  }
  if (!rc) {
    // zero everything that a kernel may read before writing
    if (cudaMemsetAsync(c->P, 0, 12 * nt * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->stats, 0, 8 * sizeof(unsigned long long), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->status, 0, na, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->iters, 0, na * sizeof(int), c->stream) != cudaSuccess)
      rc = HARMRAD_E_CUDA;
    for (int d = 0; d < 3 && !rc; ++d) {
      size_t fn = dp.n[d] > 1 ? nt : 0;
      if (fn && (cudaMemsetAsync(c->F[d], 0, 12 * fn * rs, c->stream) != cudaSuccess ||
                 cudaMemsetAsync(c->spd[d], 0, fn * rs, c->stream) != cudaSuccess ||
                 cudaMemsetAsync(c->flat[d], 0, 2 * fn * rs, c->stream) != cudaSuccess))
        rc = HARMRAD_E_CUDA;
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

void harmrad_destroy(harmrad_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  free(c);
}

int harmrad_set_prims(harmrad_ctx* c, const double* P, int on_device) {
  if (!c || !P) return HARMRAD_E_ARG;
  const DevParams& p = c->dp;
  size_t bytes = 12 * (size_t)p.nact * sizeof(double);
  const double* src = P;
  if (!on_device) {
    HR_CHECK(cudaMemcpyAsync(c->stage_buf, P, bytes, cudaMemcpyHostToDevice, c->stream));
    src = c->stage_buf;
  }
  HR_CHECK(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  int g = hr::grid_for(12 * p.nact, c->sms, 256);
  k_validate<<<g, 256, 0, c->stream>>>(p, src, c->flag);
  k_unpack<<<g, 256, 0, c->stream>>>(p, src, c->P);
  HR_CHECK(cudaGetLastError());
  int flag = 0;
  HR_CHECK(cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  if (flag) return HARMRAD_E_NAN_INPUT;
  c->has_prims = true;
  return HARMRAD_OK;
}

int harmrad_get_prims(harmrad_ctx* c, double* P, int on_device) {
  if (!c || !P) return HARMRAD_E_ARG;
  const DevParams& p = c->dp;
  size_t bytes = 12 * (size_t)p.nact * sizeof(double);
  int g = hr::grid_for(12 * p.nact, c->sms, 256);
  double* dst = on_device ? P : c->stage_buf;
  k_pack<<<g, 256, 0, c->stream>>>(p, c->P, dst);
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
  HR_CHECK(cudaMemcpyAsync(c->host_dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  *dt = *c->host_dt;
  return HARMRAD_OK;
}

int harmrad_step(harmrad_ctx* c, double dt) {
  if (!c) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  bool with_cfl = !(dt > 0.0);
  if (!with_cfl) {
    // the value travels as a kernel argument: no host synchronisation
    k_set_dt<<<1, 32, 0, c->stream>>>(c->dt, dt);
    HR_CHECK(cudaGetLastError());
  }
  c->last_dt = dt;
  return launch_step(c, with_cfl);
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
    k_set_dt<<<1, 32, 0, c->stream>>>(c->dt, dt);
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
  double dt = 0.0;
  HR_CHECK(cudaMemcpyAsync(h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaMemcpyAsync(&dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  s->dt = dt;
  s->pmhd_ok = (long long)h[hr::ST_PMHD];
  s->urad_ok = (long long)h[hr::ST_URAD];
  s->backup = (long long)h[hr::ST_BACKUP];
  s->zone_stages = (long long)h[hr::ST_SOLVES];
  s->newton_iters = (long long)h[hr::ST_ITERS];
  s->kernel_launches = c->launches_per_step;
  s->graph = c->use_graph ? 1 : 0;
  return s->backup > 0 ? HARMRAD_W_BACKUP_USED : HARMRAD_OK;
}

int harmrad_get_status(harmrad_ctx* c, unsigned char* st, int on_device) {
  if (!c || !st) return HARMRAD_E_ARG;
  HR_CHECK(cudaMemcpyAsync(st, c->status, c->dp.nact,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_get_iters(harmrad_ctx* c, int* it, int on_device) {
  if (!c || !it) return HARMRAD_E_ARG;
  HR_CHECK(cudaMemcpyAsync(it, c->iters, c->dp.nact * sizeof(int),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  HR_CHECK(cudaStreamSynchronize(c->stream));
  return HARMRAD_OK;
}

int harmrad_compute_fluxes(harmrad_ctx* c, int dir, double* F_host) {
  if (!c || !F_host || dir < 1 || dir > 3) return HARMRAD_E_ARG;
  if (!c->has_prims) return HARMRAD_E_STATE;
  const DevParams& p = c->dp;
  int d = dir - 1;
  if (p.n[d] == 1) return HARMRAD_E_ARG;
  int r = run_faces(c, true);
  if (r < 0) return r;
  size_t rs = c->real_size;
  size_t bytes = 12 * (size_t)p.ntot * rs;
  char* hbuf = (char*)malloc(bytes);
  if (!hbuf) return HARMRAD_E_OOM;
  if (cudaMemcpyAsync(hbuf, c->F[d], bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    free(hbuf);
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  int m[3] = {p.n[0], p.n[1], p.n[2]};
  m[d] += 1;
  long long nf = (long long)m[0] * m[1] * m[2];
  for (int q = 0; q < 12; ++q)
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i) {
          long long t = ((long long)(k + p.ng[2]) * p.N[1] + (j + p.ng[1])) * p.N[0] + (i + p.ng[0]);
          long long o = (long long)q * nf + ((long long)k * m[1] + j) * m[0] + i;
          F_host[o] = rs == 8 ? ((double*)hbuf)[q * p.ntot + t] : (double)((float*)hbuf)[q * p.ntot + t];
        }
  free(hbuf);
  return HARMRAD_OK;
}

int harmrad_zone_physics(const harmrad_params* prm, int n, const double* x, const double* P, double* U,
                         double* SM, double* F, double* speeds, void* stream) {
  if (!prm || n < 0 || (n > 0 && (!x || !P))) return HARMRAD_E_ARG;
  DevParams dp;
  int rc = fill_devparams(prm, dp);
  if (rc) return rc;
  if (n == 0) return HARMRAD_OK;
  int dev, sms;
  HR_CHECK(cudaGetDevice(&dev));
  HR_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int r = dp.metric == 1 ? hr::Run<hr::KS>::zone_physics(dp, n, x, P, U, SM, F, speeds, st, sms)
                         : hr::Run<hr::MINK>::zone_physics(dp, n, x, P, U, SM, F, speeds, st, sms);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(st));
  return HARMRAD_OK;
}

int harmrad_zone_implicit(const harmrad_params* prm, int n, const double* x, const double* Us,
                          const double* Ps, const double* h, double* Pout, double* eT, int* iters,
                          unsigned char* method, void* stream) {
  if (!prm || n < 0 || (n > 0 && (!x || !Us || !Ps || !h || !Pout))) return HARMRAD_E_ARG;
  DevParams dp;
  int rc = fill_devparams(prm, dp);
  if (rc) return rc;
  if (n == 0) return HARMRAD_OK;
  int dev, sms;
  HR_CHECK(cudaGetDevice(&dev));
  HR_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int r = dp.metric == 1
              ? hr::Run<hr::KS>::zone_implicit(dp, n, x, Us, Ps, h, Pout, eT, iters, method, st, sms)
              : hr::Run<hr::MINK>::zone_implicit(dp, n, x, Us, Ps, h, Pout, eT, iters, method, st, sms);
  if (r < 0) return r;
  HR_CHECK(cudaStreamSynchronize(st));
  return HARMRAD_OK;
}

const char* harmrad_strerror(int code) {
  switch (code) {
    case HARMRAD_OK: return "ok";
    case HARMRAD_W_BACKUP_USED: return "warning: some zones used the neighbour-average back-up";
    case HARMRAD_E_ARG: return "invalid argument";
    case HARMRAD_E_CUDA: return "CUDA runtime error";
    case HARMRAD_E_OOM: return "out of device memory";
    case HARMRAD_E_NAN_INPUT: return "primitives not finite or not positive";
    case HARMRAD_E_STATE: return "call out of order (no primitives loaded)";
    default: return "unknown harmrad return code";
  }
}

}  // extern "C"
