// Host sequence of the adjoint of one step (internal): recompute the step
// from its saved input with the records the reverse sweep needs, then sweep
// the sub-steps in reverse.  Instantiated per metric in hr_adj_*.cu.
#pragma once
#include "hr_adjoint.cuh"
#include "hr_run.cuh"

namespace hr {

#define HR_ACHECK(x)                 \
  do {                               \
    if ((x) != cudaSuccess) {        \
      cudaGetLastError();            \
      return HARMRAD_E_CUDA;         \
    }                                \
  } while (0)

template <int MET>
int Run<MET>::adjoint(harmrad_ctx* c, const double* gPout, double* gPin, double* gk_out) {
  const DevParams& p = c->dp;
  const BoxGeo& bx = c->boxes[0];
  const AdjBufs& a = *c->adj;
  cudaStream_t st = c->stream;
  const long long nt = bx.ntot, na = bx.nact;
  const size_t pbytes = 12 * (size_t)nt * sizeof(double);
  const int sms = c->sms;
  auto G = [&](long long work) { return grid_for(work, sms, 128); };

  // ---- recompute the step from its input, recording what the sweep needs
  HR_ACHECK(cudaMemcpyAsync(c->P, c->adj_Pn, pbytes, cudaMemcpyDeviceToDevice, st));
  for (int s = 0; s < 3; ++s) {
    HR_ACHECK(cudaMemcpyAsync(a.Pst + (size_t)s * 12 * nt, c->P, pbytes, cudaMemcpyDeviceToDevice, st));
    int r = faces_impl<MET, double>(c, s == 0);
    if (r < 0) return r;
    if (p.recon == 0)
      for (int d = 0; d < 3; ++d)
        if (p.act[d])
          HR_ACHECK(cudaMemcpyAsync(a.chi + ((size_t)s * 3 + d) * 2 * nt, c->flat[d], 2 * nt * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
    c->rec_ust = a.Ust + (size_t)s * 12 * na;
    c->rec_meth = a.meth + (size_t)s * na;
    c->rec_psol = a.Psol + (size_t)s * 12 * na;
    c->rec_sst = a.Sst + (size_t)s * na;
    r = solve_impl<MET, double>(c, s, ImexStage{});
    c->rec_ust = nullptr;
    c->rec_meth = nullptr;
    c->rec_psol = nullptr;
    c->rec_sst = nullptr;
    if (r < 0) return r;
  }
  HR_ACHECK(cudaMemcpyAsync(a.Pst + (size_t)3 * 12 * nt, c->P, pbytes, cudaMemcpyDeviceToDevice, st));

  // ---- reverse sweep
  HR_ACHECK(cudaMemcpyAsync(a.gN, gPout, 12 * (size_t)na * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HR_ACHECK(cudaMemsetAsync(a.gUn, 0, 12 * (size_t)na * sizeof(double), st));
  HR_ACHECK(cudaMemsetAsync(a.carry, 0, 6 * (size_t)nt * sizeof(double), st));
  HR_ACHECK(cudaMemsetAsync(a.gk, 0, sizeof(double), st));
  HR_ACHECK(cudaMemsetAsync(a.gSn, 0, (size_t)na * sizeof(double), st));
  // a zone solved by the cold-MHD equations (its u_g the neighbours'
  // average) has no adjoint here: the step is refused
  HR_ACHECK(cudaMemsetAsync(c->flag, 0, sizeof(int), st));
  ka_find_meth<<<G(3 * na), 128, 0, st>>>(a.meth, 3 * na, METH_COLD, c->flag);
  double dt = 0.0;
  int cold = 0;
  HR_ACHECK(cudaMemcpyAsync(&dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, st));
  HR_ACHECK(cudaMemcpyAsync(&cold, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HR_ACHECK(cudaStreamSynchronize(st));
  if (cold) return HARMRAD_E_ARG;
  const double* K = c->K;
  double* aux = (double*)c->aux;
  double* Pg = c->P;
  for (int s = 2; s >= 0; --s) {
    const double* Pnext = a.Pst + (size_t)(s + 1) * 12 * nt;
    const double* Ps = a.Pst + (size_t)s * 12 * nt;
    ka_backup_T<<<G(na), 128, 0, st>>>(bx, a.meth + (size_t)s * na, a.gN);
    ka_implicit<MET><<<G(na), 128, 0, st>>>(p, bx, a, s, dt, K, Pnext);
    // forward state of the sub-step: P_s with ghosts, cell factors
    HR_ACHECK(cudaMemcpyAsync(Pg, Ps, pbytes, cudaMemcpyDeviceToDevice, st));
    for (int d = 0; d < 3; ++d) {
      if (!p.act[d]) continue;
      long long work = 2LL * bx.ng[d];
      for (int e = 0; e < 3; ++e)
        if (e != d) work *= (e < d) ? bx.N[e] : bx.n[e];
      k_bc_fill<<<G(work), 128, 0, st>>>(p, c->dboxes, 1, Pg, p.opacity == 2 ? c->K : nullptr, d);
    }
    k_prep<MET, double><<<G(nt), 128, 0, st>>>(p, c->dboxes, 1, Pg, c->K, aux, c->geotab);
    HR_ACHECK(cudaMemsetAsync(a.gP, 0, pbytes, st));
    ka_update<MET><<<G(na), 128, 0, st>>>(p, bx, a, s, dt, Ps);
    // fluxes: divergence, then flux-CT
    for (int d = 0; d < 3; ++d) {
      if (!p.act[d]) continue;
      long long w = 1;
      for (int e = 0; e < 3; ++e) w *= (e == d) ? bx.n[e] + 1 : (bx.n[e] > 1 ? bx.n[e] + 2 : 1);
      if (d == 0) ka_fluxgrad<0><<<G(w), 128, 0, st>>>(bx, a.gX, a.gF[0], a.gXS, a.gFS[0]);
      if (d == 1) ka_fluxgrad<1><<<G(w), 128, 0, st>>>(bx, a.gX, a.gF[1], a.gXS, a.gFS[1]);
      if (d == 2) ka_fluxgrad<2><<<G(w), 128, 0, st>>>(bx, a.gX, a.gF[2], a.gXS, a.gFS[2]);
    }
    for (int pa = 0; pa < 3; ++pa)
      for (int pb = pa + 1; pb < 3; ++pb) {
        if (!p.act[pa] || !p.act[pb]) continue;
        long long we = 1;
        for (int e = 0; e < 3; ++e) we *= bx.n[e] + ((e == pa || e == pb) ? 1 : 0);
        double* gFab = a.gF[pa] + (size_t)(B1 + pb) * nt;
        double* gFba = a.gF[pb] + (size_t)(B1 + pa) * nt;
        ka_emf_T<<<G(we), 128, 0, st>>>(p, bx, gFab, gFba, a.gemf, pa, pb);
        auto faces_of = [&](int d) {
          long long w = 1;
          for (int e = 0; e < 3; ++e) w *= (e == d) ? bx.n[e] + 1 : (bx.n[e] > 1 ? bx.n[e] + 2 : 1);
          return w;
        };
        if (pa == 0) ka_ct_T<0><<<G(faces_of(0)), 128, 0, st>>>(bx, a.gemf, gFab, pb, 1.0);
        if (pa == 1) ka_ct_T<1><<<G(faces_of(1)), 128, 0, st>>>(bx, a.gemf, gFab, pb, 1.0);
        if (pb == 1) ka_ct_T<1><<<G(faces_of(1)), 128, 0, st>>>(bx, a.gemf, gFba, pa, -1.0);
        if (pb == 2) ka_ct_T<2><<<G(faces_of(2)), 128, 0, st>>>(bx, a.gemf, gFba, pa, -1.0);
      }
    // per direction: reconstruction and Riemann fluxes, flattener, cell factors
    for (int d = 0; d < 3; ++d) {
      if (!p.act[d]) continue;
      long long wf = 1, wc = 1, ws = 1;
      for (int e = 0; e < 3; ++e) {
        wf *= (e == d) ? bx.n[e] + 1 : (bx.n[e] > 1 ? bx.n[e] + 2 : 1);
        wc *= bx.n[e] > 1 ? bx.n[e] + 2 : 1;
        ws *= bx.n[e] > 1 ? bx.n[e] + (e == d ? 4 : 2) : 1;
      }
      const double* chi_s = a.chi + ((size_t)s * 3 + d) * 2 * nt;
      const double* chi_prev = s > 0 ? a.chi + ((size_t)(s - 1) * 3 + d) * 2 * nt : nullptr;
      double* E = (double*)c->edges;
      double* carry = a.carry + (size_t)d * 2 * nt;
      HR_ACHECK(cudaMemsetAsync(a.gE, 0, 24 * (size_t)nt * sizeof(double), st));
      HR_ACHECK(cudaMemsetAsync(a.gaux, 0, 3 * (size_t)nt * sizeof(double), st));
      const double* flat = p.recon == 0 ? chi_s : aux;  // not read for MC
      if (d == 0) {
        k_slopes<MET, double, 0><<<G(ws), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, (double*)c->slope);
        k_edges<MET, double, 0><<<G(wc), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, flat, (double*)c->slope, E);
        ka_face<MET, 0><<<G(wf), 128, 0, st>>>(p, bx, E, K, a.gF[0], a.gE, a.gk, a.gFS[0]);
        ka_edges<MET, 0><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, flat, a.gE, a.gP, a.gchi);
        if (p.recon == 0) {
          ka_flatten<0><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, chi_prev, a.gchi, carry, a.gP, a.gaux);
          ka_prep<MET, 0><<<G(nt), 128, 0, st>>>(p, bx, Pg, K, a.gaux, a.gP, a.gk);
        }
      } else if (d == 1) {
        k_slopes<MET, double, 1><<<G(ws), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, (double*)c->slope);
        k_edges<MET, double, 1><<<G(wc), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, flat, (double*)c->slope, E);
        ka_face<MET, 1><<<G(wf), 128, 0, st>>>(p, bx, E, K, a.gF[1], a.gE, a.gk, a.gFS[1]);
        ka_edges<MET, 1><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, flat, a.gE, a.gP, a.gchi);
        if (p.recon == 0) {
          ka_flatten<1><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, chi_prev, a.gchi, carry, a.gP, a.gaux);
          ka_prep<MET, 1><<<G(nt), 128, 0, st>>>(p, bx, Pg, K, a.gaux, a.gP, a.gk);
        }
      } else {
        k_slopes<MET, double, 2><<<G(ws), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, (double*)c->slope);
        k_edges<MET, double, 2><<<G(wc), 128, 0, st>>>(p, c->dboxes, 1, Pg, aux, flat, (double*)c->slope, E);
        ka_face<MET, 2><<<G(wf), 128, 0, st>>>(p, bx, E, K, a.gF[2], a.gE, a.gk, a.gFS[2]);
        ka_edges<MET, 2><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, flat, a.gE, a.gP, a.gchi);
        if (p.recon == 0) {
          ka_flatten<2><<<G(wc), 128, 0, st>>>(p, bx, Pg, aux, chi_prev, a.gchi, carry, a.gP, a.gaux);
          ka_prep<MET, 2><<<G(nt), 128, 0, st>>>(p, bx, Pg, K, a.gaux, a.gP, a.gk);
        }
      }
    }
    // ghost fill, reverse order of directions
    for (int d = 2; d >= 0; --d) {
      if (!p.act[d]) continue;
      long long work = 2LL * bx.ng[d];
      for (int e = 0; e < 3; ++e)
        if (e != d) work *= (e < d) ? bx.N[e] : bx.n[e];
      ka_bc_T<<<G(work), 128, 0, st>>>(bx, Pg, a.gP, d);
    }
    ka_gather<<<G(na), 128, 0, st>>>(bx, a.gP, a.gN);
    HR_ACHECK(cudaGetLastError());
  }
  // U^n = U(P^n)
  ka_un<MET><<<G(na), 128, 0, st>>>(p, bx, a, a.Pst);
  HR_ACHECK(cudaGetLastError());
  HR_ACHECK(cudaMemcpyAsync(gPin, a.gN, 12 * (size_t)na * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (gk_out) HR_ACHECK(cudaMemcpyAsync(gk_out, a.gk, sizeof(double), cudaMemcpyDeviceToDevice, st));
  // leave the state of the step's end in place
  HR_ACHECK(cudaMemcpyAsync(c->P, a.Pst + (size_t)3 * 12 * nt, pbytes, cudaMemcpyDeviceToDevice, st));
  return HARMRAD_OK;
}

#undef HR_ACHECK

}  // namespace hr
