// Adjoint (reverse-mode derivative) of one full RK3 step, FP64, one grid.
//
// The reverse sweep visits the sub-steps of Sec. 4.1-4.2 in reverse order and,
// inside each, the operations of the sub-step in reverse: implicit solve,
// explicit update, flux-CT, Riemann fluxes, reconstruction, flattener, cell
// factors and ghost fill.  Each kernel applies the transpose of its forward
// operation's local Jacobian to the incoming cotangent; the local Jacobians
// come from evaluating the forward device functions on dual numbers (Dn<N>),
// so every branch (limiters, wave-speed maxima, flattener clamps) takes the
// derivative of the branch the forward step took.
//
// The implicit solve is differentiated through its solution, not through the
// Newton iterations (implicit-function theorem): at the root x* of the PMHD
// error E(x; U*, kappa) = 0, dx*/dU* = -J_x^{-1} dE/dU*, so the cotangent of
// U* is  gU = (dP/dU*)^T gP - (dE/dU*)^T lambda  with  J_x^T lambda = (dP/dx)^T gP,
// one transposed 4x4 solve per zone.  The floors act on the solution: their
// Jacobian (identity for the components they leave alone, the derivative of
// the floor value for those they set) is applied first.  Zones that took the
// neighbour-average back-up pass their cotangent to the neighbours they
// averaged (B, which is U*[B]/sqrt(-g), excepted).  The time step is held
// fixed.
#pragma once
#include "hr_kernels.cuh"

namespace hr {

struct AdjBufs {
  double* Pst;          // [4][12][ntot] sub-step inputs P_0, P_1, P_2 and the result P^{n+1}
  double* chi;          // [3][3][2][ntot] flattener after sub-step s, per direction (PPM)
  double* Ust;          // [3][12][nact] U* of every zone and sub-step
  unsigned char* meth;  // [3][nact] outcome per sub-step: 0 PMHD, 1 URAD, 2 back-up, 3 entropy
  double* Psol;         // [3][12][nact] solution of every zone before the floors
  double* gP;           // [12][ntot] cotangent of the current sub-step's input (ghosts included)
  double* gN;           // [12][nact] cotangent of the current sub-step's output
  double* gUn;          // [12][nact] cotangent of U^n
  double* gU;           // [12][nact] cotangent of U*
  double* gX;           // [12][nact] cotangent of the explicit rate X
  double* gF[3];        // [12][ntot] cotangent of the face fluxes
  double* gE;           // [24][ntot] cotangent of the reconstructed edges of one direction
  double* gchi;         // [2][ntot] cotangent of the flattener used by one direction's edges
  double* carry;        // [3][2][ntot] flattener cotangent passed to the earlier sub-step
  double* gaux;         // [3][ntot] cotangent of sqrt(-g) u^d (gas, rad) and w_d of one direction
  double* gemf;         // [ntot] cotangent of the edge EMFs of one pair of directions
  double* gk;           // [1] cotangent of kappa_scale
  // the entropy (Sec. 2, Eq. S), for zones solved by the entropy equation
  double* Sst;          // [3][nact] explicit entropy S* of every zone and sub-step
  double* gS;           // [nact] cotangent of S*
  double* gSn;          // [nact] cotangent of S^n, the step's initial conserved entropy
  double* gXS;          // [nact] cotangent of the entropy's explicit rate X_S = -div F_S
  double* gFS[3];       // [ntot] cotangent of the entropy face fluxes
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Adds v of every lane of a full warp to *dst (one atomic per warp).  Called
// by all 32 lanes (no early exit between the grid-stride loop and this call).
__device__ __forceinline__ void warp_atomic_add(double* dst, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

__device__ __forceinline__ void zone_ijk(const BoxGeo& bx, long long z, int& i, int& j, int& k) {
  long long r = z;
  i = (int)(r % bx.n[0]);
  r /= bx.n[0];
  j = (int)(r % bx.n[1]);
  k = (int)(r / bx.n[1]);
}

__device__ __forceinline__ long long zone_of(const BoxGeo& bx, int i, int j, int k) {
  return ((long long)k * bx.n[1] + j) * bx.n[0] + i;
}

// Sets *flag when any of the n method records equals m.
static __global__ void ka_find_meth(const unsigned char* __restrict__ meth, long long n, unsigned char m, int* flag) {
  for (long long z = HR_TID; z < n; z += HR_STRIDE)
    if (meth[z] == m) *flag = 1;
}

// ------------------------------------------------------------ back-up (T)
// A back-up zone's non-B primitives are the average of its good neighbours'
// solutions: its cotangent moves to those neighbours.
static __global__ void ka_backup_T(BoxGeo bx, const unsigned char* __restrict__ meth, double* gN) {
  for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
    if (meth[z] != 2) continue;
    int ii[3];
    zone_ijk(bx, z, ii[0], ii[1], ii[2]);
    long long nb_z[6];
    int ng = 0;
    for (int d = 0; d < 3; ++d) {
      if (bx.n[d] == 1) continue;
      for (int side = -1; side <= 1; side += 2) {
        int nb[3] = {ii[0], ii[1], ii[2]};
        nb[d] += side;
        if (nb[d] < 0 || nb[d] >= bx.n[d]) continue;
        long long zn = zone_of(bx, nb[0], nb[1], nb[2]);
        if (meth[zn] != 2) nb_z[ng++] = zn;
      }
    }
    for (int q = 0; q < NPR; ++q) {
      if (q >= B1 && q <= B3) continue;
      double g = gN[q * bx.nact + z];
      gN[q * bx.nact + z] = 0.0;
      if (ng == 0 || g == 0.0) continue;
      g /= ng;
      for (int e = 0; e < ng; ++e) atomicAdd(&gN[q * bx.nact + nb_z[e]], g);
    }
  }
}

// ------------------------------------------------------- implicit solve (T)
template <int MET>
__global__ void ka_implicit(DevParams p, BoxGeo bx, AdjBufs a, int s, double dt, const double* __restrict__ K,
                            const double* __restrict__ Pnext) {
  const double Bc = s == 0 ? 1.0 : (s == 1 ? 0.25 : 2.0 / 3.0);
  const double h = Bc * dt;
  const double* Ust0 = a.Ust + (long long)s * 12 * bx.nact;
  const unsigned char* meth = a.meth + (long long)s * bx.nact;
  const double* Psol0 = a.Psol + (long long)s * 12 * bx.nact;
  typedef Dn<4> D4;
  typedef Dn<1> D1;
  double gk = 0.0;
  for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
    double gq[NPR];
    bool any = false;
    for (int q = 0; q < NPR; ++q) {
      gq[q] = a.gN[q * bx.nact + z];
      any = any || gq[q] != 0.0;
      a.gU[q * bx.nact + z] = 0.0;
    }
    a.gS[z] = 0.0;
    if (!any) continue;
    int i, j, k;
    zone_ijk(bx, z, i, j, k);
    const long long t = cell_index(bx, i, j, k);
    const double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
    const Geo<MET, double> g = make_geo<MET, double>(p, x1, x2);
    const double igd = 1.0 / g.gdet;
    const int m = meth[z];
    double Us[NPR], Ps[NPR];
    for (int q = 0; q < NPR; ++q) {
      Us[q] = Ust0[q * bx.nact + z];
      Ps[q] = Psol0[q * bx.nact + z];
    }
    (void)Pnext;
    const double kz = kfield(p, K, t);
    if (m == 2) {  // back-up: only B = U*[B] / sqrt(-g) is the zone's own
      for (int c = 0; c < 3; ++c) a.gU[(B1 + c) * bx.nact + z] = gq[B1 + c] * igd;
      continue;
    }
    // a zone solved by the entropy equation (by the entropy PMHD, URAD or
    // PRAD, which solve the same equations): the same transposed solve on the
    // entropy system (Eq. source6), which also depends on S*
    const bool ent = m == METH_ENTROPY;
    const double Sz = ent ? a.Sst[(long long)s * bx.nact + z] : 0.0;
    const Geo<MET, D4> g4 = geo_cast<D4>(g);
    {  // floors: gq <- (d floors / d P)^T gq at the solution
      const double rr = log_r<MET>(p, x1);
      double gs[NPR];
      for (int ch = 0; ch < 3; ++ch) {
        D4 PD[NPR];
        for (int q = 0; q < NPR; ++q) PD[q] = D4::seed(Ps[q], q - 4 * ch);
        apply_floors<MET, D4>(p, g4, rr, PD);
        for (int c = 0; c < 4; ++c) {
          double v = 0.0;
          for (int q = 0; q < NPR; ++q) v += gq[q] * PD[q].d[c];
          gs[4 * ch + c] = v;
        }
      }
      for (int q = 0; q < NPR; ++q) gq[q] = gs[q];
    }
    const double x[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
    double J[4][4], gx[4] = {0.0, 0.0, 0.0, 0.0};
    {  // derivatives with respect to x
      D4 xs[4], UsD[NPR], PsD[NPR], Eg[4];
      for (int c = 0; c < 4; ++c) xs[c] = D4::seed(x[c], c);
      for (int q = 0; q < NPR; ++q) UsD[q] = D4(Us[q]);
      ImpSysT<MET, D4> sys;
      build_sys<MET, D4>(p, g4, UsD, h, D4(kz), sys);
      sys.entropy = ent;
      sys.Sstar = D4(Sz * igd);
      pmhd_final<MET, D4>(p, sys, xs, PsD, Eg);
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) J[c][r] = Eg[r].d[c];  // transposed
      for (int q = 0; q < NPR; ++q)
        for (int c = 0; c < 4; ++c) gx[c] += gq[q] * PsD[q].d[c];
    }
    double lam[4];
    if (!solve4(J, gx, lam)) continue;
    double gU[NPR];
    for (int ch = 0; ch < 3; ++ch) {  // derivatives with respect to U*, four at a time
      D4 xs[4], UsD[NPR], PsD[NPR], Eg[4];
      for (int c = 0; c < 4; ++c) xs[c] = D4(x[c]);
      for (int q = 0; q < NPR; ++q) UsD[q] = D4::seed(Us[q], q - 4 * ch);
      ImpSysT<MET, D4> sys;
      build_sys<MET, D4>(p, g4, UsD, h, D4(kz), sys);
      sys.entropy = ent;
      sys.Sstar = D4(Sz * igd);
      pmhd_final<MET, D4>(p, sys, xs, PsD, Eg);
      for (int c = 0; c < 4; ++c) {
        double v = 0.0;
        for (int q = 0; q < NPR; ++q) v += gq[q] * PsD[q].d[c];
        for (int r = 0; r < 4; ++r) v -= lam[r] * Eg[r].d[c];
        gU[4 * ch + c] = v;
      }
    }
    {  // derivative with respect to kappa_scale (E only; P depends on it through x*)
      const Geo<MET, D1> g1 = geo_cast<D1>(g);
      D1 xs[4], UsD[NPR], PsD[NPR], Eg[4];
      for (int c = 0; c < 4; ++c) xs[c] = D1(x[c]);
      for (int q = 0; q < NPR; ++q) UsD[q] = D1(Us[q]);
      ImpSysT<MET, D1> sys;
      build_sys<MET, D1>(p, g1, UsD, h, D1(kz), sys);
      sys.ks = D1::seed(p.kscale, 0);
      sys.entropy = ent;
      sys.Sstar = D1(Sz * igd);
      pmhd_final<MET, D1>(p, sys, xs, PsD, Eg);
      for (int r = 0; r < 4; ++r) gk -= lam[r] * Eg[r].d[0];
    }
    for (int q = 0; q < NPR; ++q) a.gU[q * bx.nact + z] = gU[q];
    // S* enters the entropy row only, E_0 = T (S u^t(x) - S*/sqrt(-g)) +
    // h G_mu u^mu with T = p/rho0 at the solution (the factor F_13)
    if (ent) a.gS[z] = lam[0] * ((p.gam - 1.0) * Ps[UU] / Ps[RHO]) * igd;
  }
  warp_atomic_add(a.gk, gk);
}

// --------------------------------------------------- explicit update (T)
// U* = a_s U^n + b_s (U(P_s) + dt X),  X = -sum_d dF_d/dx_d + SM(P_s).
template <int MET>
__global__ void ka_update(DevParams p, BoxGeo bx, AdjBufs a, int s, double dt, const double* __restrict__ Ps0) {
  const double A = s == 0 ? 0.0 : (s == 1 ? 0.75 : 1.0 / 3.0);
  const double Bc = s == 0 ? 1.0 : (s == 1 ? 0.25 : 2.0 / 3.0);
  typedef Dn<4> D4;
  for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
    double gq[NPR];
    bool any = false;
    for (int q = 0; q < NPR; ++q) {
      gq[q] = a.gU[q * bx.nact + z];
      any = any || gq[q] != 0.0;
      if (s > 0) a.gUn[q * bx.nact + z] += A * gq[q];
      a.gX[q * bx.nact + z] = Bc * dt * gq[q];
    }
    // S* = A S^n + Bc (S(P_s) + dt X_S), S(P) = U_rho(P) s_gas(P)
    const double gs = a.gS[z];
    any = any || gs != 0.0;
    if (s > 0) a.gSn[z] += A * gs;
    a.gXS[z] = Bc * dt * gs;
    int i, j, k;
    zone_ijk(bx, z, i, j, k);
    const long long t = cell_index(bx, i, j, k);
    if (!any) {
      for (int q = 0; q < NPR; ++q) a.gP[q * bx.ntot + t] = 0.0;
      continue;
    }
    const double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
    const Geo<MET, D4> g4 = geo_cast<D4>(make_geo<MET, double>(p, x1, x2));
    for (int ch = 0; ch < 3; ++ch) {
      D4 PsD[NPR], UsD[NPR], XD[NPR];
      for (int q = 0; q < NPR; ++q) PsD[q] = D4::seed(Ps0[q * bx.ntot + t], q - 4 * ch);
      cons_source<MET, D4>(p, g4, x1, x2, PsD, UsD, XD);
      const D4 Su = gs != 0.0 ? UsD[RHO] * entropy_per_baryon<D4>(p, PsD[RHO], PsD[UU]) : D4(0.0);
      for (int c = 0; c < 4; ++c) {
        double v = gs * Su.d[c];
        for (int q = 0; q < NPR; ++q) v += gq[q] * (UsD[q].d[c] + dt * XD[q].d[c]);
        a.gP[(4 * ch + c) * bx.ntot + t] = Bc * v;
      }
    }
  }
}

// U^n = U(P^n): gP^n += (dU/dP)^T gU^n at the end of the sweep.
template <int MET>
__global__ void ka_un(DevParams p, BoxGeo bx, AdjBufs a, const double* __restrict__ P0) {
  typedef Dn<4> D4;
  for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
    double gq[NPR];
    bool any = false;
    for (int q = 0; q < NPR; ++q) {
      gq[q] = a.gUn[q * bx.nact + z];
      any = any || gq[q] != 0.0;
    }
    const double gs = a.gSn[z];  // S^n = U_rho(P^n) s_gas(P^n)
    any = any || gs != 0.0;
    if (!any) continue;
    int i, j, k;
    zone_ijk(bx, z, i, j, k);
    const long long t = cell_index(bx, i, j, k);
    const double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
    const Geo<MET, D4> g4 = geo_cast<D4>(make_geo<MET, double>(p, x1, x2));
    for (int ch = 0; ch < 3; ++ch) {
      D4 PsD[NPR], UsD[NPR], XD[NPR];
      for (int q = 0; q < NPR; ++q) PsD[q] = D4::seed(P0[q * bx.ntot + t], q - 4 * ch);
      cons_source<MET, D4>(p, g4, x1, x2, PsD, UsD, XD);
      const D4 Su = gs != 0.0 ? UsD[RHO] * entropy_per_baryon<D4>(p, PsD[RHO], PsD[UU]) : D4(0.0);
      for (int c = 0; c < 4; ++c) {
        double v = gs * Su.d[c];
        for (int q = 0; q < NPR; ++q) v += gq[q] * UsD[q].d[c];
        a.gN[(4 * ch + c) * bx.nact + z] += v;
      }
    }
  }
}

// ------------------------------------------------ flux divergence (T)
// Face range of the face kernel of direction d; the flux at cell t is the
// flux through t's lower face: +1/dx in X of zone t, -1/dx in X of zone t-s_d.
template <int d>
__global__ void ka_fluxgrad(BoxGeo bx, const double* __restrict__ gX, double* __restrict__ gF,
                            const double* __restrict__ gXS, double* __restrict__ gFS) {
  int len[3], off[3];
  for (int e = 0; e < 3; ++e) {
    if (e == d) {
      len[e] = bx.n[e] + 1;
      off[e] = 0;
    } else if (bx.n[e] > 1) {
      len[e] = bx.n[e] + 2;
      off[e] = -1;
    } else {
      len[e] = 1;
      off[e] = 0;
    }
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const double idx_ = 1.0 / bx.dx[d];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int ii[3];
    ii[0] = (int)(r % len[0]) + off[0];
    r /= len[0];
    ii[1] = (int)(r % len[1]) + off[1];
    ii[2] = (int)(r / len[1]) + off[2];
    const long long t = cell_index(bx, ii[0], ii[1], ii[2]);
    bool trans = true;
    for (int e = 0; e < 3; ++e)
      if (e != d && (ii[e] < 0 || ii[e] >= bx.n[e])) trans = false;
    const int f = ii[d];
    const bool up = trans && f < bx.n[d];
    const bool dn = trans && f >= 1;
    int lo[3] = {ii[0], ii[1], ii[2]};
    lo[d] -= 1;
    const long long zu = up ? zone_of(bx, ii[0], ii[1], ii[2]) : 0;
    const long long zd = dn ? zone_of(bx, lo[0], lo[1], lo[2]) : 0;
    for (int q = 0; q < NPR; ++q) {
      double v = 0.0;
      if (up) v += gX[q * bx.nact + zu] * idx_;
      if (dn) v -= gX[q * bx.nact + zd] * idx_;
      gF[q * bx.ntot + t] = v;
    }
    if (gFS) {  // the entropy flux, X_S = -div F_S
      double v = 0.0;
      if (up) v += gXS[zu] * idx_;
      if (dn) v -= gXS[zd] * idx_;
      gFS[t] = v;
    }
  }
}

// ----------------------------------------------------------- flux-CT (T)
__device__ __forceinline__ bool in_range(const int ii[3], const int len[3]) {
  return ii[0] >= 0 && ii[0] < len[0] && ii[1] >= 0 && ii[1] < len[1] && ii[2] >= 0 && ii[2] < len[2];
}

// gEMF at every edge from the cotangents of the CT-replaced face fluxes.
static __global__ void ka_emf_T(DevParams p, BoxGeo bx, const double* __restrict__ gFab,
                                const double* __restrict__ gFba, double* __restrict__ gemf, int a, int b) {
  int len[3], la[3], lb[3];
  for (int e = 0; e < 3; ++e) {
    len[e] = bx.n[e] + ((e == a || e == b) ? 1 : 0);
    la[e] = bx.n[e] + (e == a ? 1 : 0);
    lb[e] = bx.n[e] + (e == b ? 1 : 0);
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const long long sa = bx.str[a], sb = bx.str[b];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int ii[3];
    ii[0] = (int)(r % len[0]);
    r /= len[0];
    ii[1] = (int)(r % len[1]);
    ii[2] = (int)(r / len[1]);
    const long long t = cell_index(bx, ii[0], ii[1], ii[2]);
    const bool pole = p.metric == KS && (a == 1 || b == 1) &&
                      ((ii[1] == 0 && bx.bc[2] == 2) || (ii[1] == bx.n[1] && bx.bc[3] == 2));
    double v = 0.0;
    if (!pole) {
      int m[3] = {ii[0], ii[1], ii[2]};
      if (in_range(m, la)) v += 0.5 * gFab[t];
      m[b] -= 1;
      if (in_range(m, la)) v += 0.5 * gFab[t - sb];
      m[b] += 1;
      if (in_range(m, lb)) v -= 0.5 * gFba[t];
      m[a] -= 1;
      if (in_range(m, lb)) v -= 0.5 * gFba[t - sa];
    }
    gemf[t] = v;
  }
}

// Cotangents of the Godunov induction fluxes F_a[B_b] (and F_b[B_a]) over the
// face kernel's range: their only use is the edge EMFs.
template <int dd>
__global__ void ka_ct_T(BoxGeo bx, const double* __restrict__ gemf, double* __restrict__ gFq, int other,
                        double sign) {
  int len[3], off[3], le[3];
  for (int e = 0; e < 3; ++e) {
    if (e == dd) {
      len[e] = bx.n[e] + 1;
      off[e] = 0;
    } else if (bx.n[e] > 1) {
      len[e] = bx.n[e] + 2;
      off[e] = -1;
    } else {
      len[e] = 1;
      off[e] = 0;
    }
    le[e] = bx.n[e] + ((e == dd || e == other) ? 1 : 0);
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const long long so = bx.str[other];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int ii[3];
    ii[0] = (int)(r % len[0]) + off[0];
    r /= len[0];
    ii[1] = (int)(r % len[1]) + off[1];
    ii[2] = (int)(r / len[1]) + off[2];
    const long long t = cell_index(bx, ii[0], ii[1], ii[2]);
    double v = 0.0;
    if (in_range(ii, le)) v += gemf[t];
    int m[3] = {ii[0], ii[1], ii[2]};
    m[other] += 1;
    if (in_range(m, le)) v += gemf[t + so];
    gFq[t] = sign * 0.25 * v;
  }
}

// ------------------------------------------------------ Riemann fluxes (T)
// Per face: cotangents of the two reconstructed states from the flux's
// cotangent (25 inputs: P_L, P_R, kappa_scale; five dual passes).
template <int MET, int d>
__global__ void __launch_bounds__(128) ka_face(DevParams p, BoxGeo bx, const double* __restrict__ E,
                                               const double* __restrict__ K, const double* __restrict__ gF,
                                               double* __restrict__ gE, double* gk_out,
                                               const double* __restrict__ gFS) {
  typedef Dn<5> D5;
  const bool weighted = (MET == KS) && (d != 1);
  int len[3], off[3];
  for (int e = 0; e < 3; ++e) {
    if (e == d) {
      len[e] = bx.n[e] + 1;
      off[e] = 0;
    } else if (bx.n[e] > 1) {
      len[e] = bx.n[e] + 2;
      off[e] = -1;
    } else {
      len[e] = 1;
      off[e] = 0;
    }
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const long long st = bx.str[d];
  double gk = 0.0;
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int ii[3];
    ii[0] = (int)(r % len[0]) + off[0];
    r /= len[0];
    ii[1] = (int)(r % len[1]) + off[1];
    ii[2] = (int)(r / len[1]) + off[2];
    const long long t = cell_index(bx, ii[0], ii[1], ii[2]);
    const int f = ii[d];
    if (MET == KS && d == 1 && ((f == 0 && bx.bc[2] == 2) || (f == bx.n[1] && bx.bc[3] == 2))) continue;
    double gq[NPR];
    bool any = false;
    for (int q = 0; q < NPR; ++q) {
      gq[q] = gF[q * bx.ntot + t];
      any = any || gq[q] != 0.0;
    }
    const double gfs = gFS ? gFS[t] : 0.0;
    any = any || gfs != 0.0;
    if (!any) continue;
    double xf[3];
    for (int e = 0; e < 3; ++e) xf[e] = bx.x0[e] + (ii[e] + (e == d ? 0.0 : 0.5)) * bx.dx[e];
    const Geo<MET, double> g = make_geo<MET, double>(p, xf[0], xf[1]);
    const double igf = weighted ? 1.0 / g.gdet : 1.0;
    double PL[NPR], PR[NPR], wL[NPR];
    for (int q = 0; q < NPR; ++q) {
      const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
      const double aR = E[(NPR + q) * bx.ntot + t - st];
      const double bL = E[q * bx.ntot + t];
      PL[q] = wq ? aR * igf : aR;
      PR[q] = wq ? bL * igf : bL;
      wL[q] = wq ? igf : 1.0;
    }
    const double kL = kfield(p, K, t - st), kR = kfield(p, K, t);
    const Geo<MET, D5> g5 = geo_cast<D5>(g);
    double gin[25];
    for (int ch = 0; ch < 5; ++ch) {
      D5 PLd[NPR], PRd[NPR], out[NPR], smax;
      for (int q = 0; q < NPR; ++q) {
        PLd[q] = D5::seed(PL[q], q - 5 * ch);
        PRd[q] = D5::seed(PR[q], NPR + q - 5 * ch);
      }
      const D5 ks = D5::seed(p.kscale, 24 - 5 * ch);
      D5 fs;
      face_flux<MET, D5, d>(p, g5, D5(bx.dx[d]), D5(kL), D5(kR), ks, PLd, PRd, out, &smax, nullptr,
                            gfs != 0.0 ? &fs : nullptr);
      for (int c = 0; c < 5; ++c) {
        double v = gfs != 0.0 ? gfs * fs.d[c] : 0.0;
        for (int q = 0; q < NPR; ++q) v += gq[q] * out[q].d[c];
        gin[5 * ch + c] = v;
      }
    }
    for (int q = 0; q < NPR; ++q) {
      gE[(NPR + q) * bx.ntot + t - st] = gin[q] * wL[q];  // upper edge of cell f-1
      gE[q * bx.ntot + t] = gin[NPR + q] * wL[q];         // lower edge of cell f
    }
    gk += gin[24];
  }
  warp_atomic_add(gk_out, gk);
}

// ----------------------------------------------------- reconstruction (T)
// Per cell of the edge range: cotangents of the five stencil primitives of
// every variable (atomic, the stencils overlap) and of the cell's flattener.
template <int MET, int d>
__global__ void ka_edges(DevParams p, BoxGeo bx, const double* __restrict__ P, const double* __restrict__ aux,
                         const double* __restrict__ flat, const double* __restrict__ gE, double* gP,
                         double* __restrict__ gchi) {
  typedef Dn<6> D6;
  const bool weighted = (MET == KS) && (d != 1);
  int len[3], off[3];
  for (int e = 0; e < 3; ++e) {
    if (bx.n[e] > 1) {
      len[e] = bx.n[e] + 2;
      off[e] = -1;
    } else {
      len[e] = 1;
      off[e] = 0;
    }
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const long long st = bx.str[d];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int i = (int)(r % len[0]) + off[0];
    r /= len[0];
    int j = (int)(r % len[1]) + off[1];
    int k = (int)(r / len[1]) + off[2];
    const long long t = cell_index(bx, i, j, k);
    double gcg = 0.0, gcr = 0.0;
    const double chg = p.recon == 0 ? flat[t] : 0.0, chr = p.recon == 0 ? flat[bx.ntot + t] : 0.0;
    double gw[5];
    for (int m = 0; m < 5; ++m) gw[m] = weighted ? aux[t + (m - 2) * st] : 1.0;
    for (int q = 0; q < NPR; ++q) {
      const double gl = gE[q * bx.ntot + t], gr = gE[(NPR + q) * bx.ntot + t];
      if (gl == 0.0 && gr == 0.0) continue;
      const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
      D6 sD[5];
      for (int m = 0; m < 5; ++m) {
        const double v = P[q * bx.ntot + t + (m - 2) * st];
        sD[m] = D6::seed(wq ? gw[m] * v : v, m);
      }
      D6 aL, aR;
      if (p.recon == 0) {
        D6 chi = D6::seed(q < ER ? chg : chr, 5);
        ppm_cell<D6>(sD, chi, &aL, &aR);
      } else {
        D6 dq = mc_slope<D6>(sD[1], sD[2], sD[3]);
        aL = sD[2] - 0.5 * dq;
        aR = sD[2] + 0.5 * dq;
      }
      for (int m = 0; m < 5; ++m) {
        const double v = gl * aL.d[m] + gr * aR.d[m];
        if (v != 0.0) atomicAdd(&gP[q * bx.ntot + t + (m - 2) * st], wq ? v * gw[m] : v);
      }
      const double vc = gl * aL.d[5] + gr * aR.d[5];
      if (q < ER) gcg += vc;
      else gcr += vc;
    }
    gchi[t] = gcg;
    gchi[bx.ntot + t] = gcr;
  }
}

// ---------------------------------------------------------- flattener (T)
// The flattener after sub-step s is max(previous, new); the cotangent goes to
// the new value where it won (strictly greater, as in the forward), else it
// is carried to the earlier sub-step.
template <int d>
__global__ void ka_flatten(DevParams p, BoxGeo bx, const double* __restrict__ P, const double* __restrict__ aux,
                           const double* __restrict__ prev, const double* __restrict__ gchi, double* carry,
                           double* gP, double* gaux) {
  typedef Dn<5> D5;
  int len[3], off[3];
  for (int e = 0; e < 3; ++e) {
    if (bx.n[e] > 1) {
      len[e] = bx.n[e] + 2;
      off[e] = -1;
    } else {
      len[e] = 1;
      off[e] = 0;
    }
  }
  const long long total = (long long)len[0] * len[1] * len[2];
  const long long st = bx.str[d];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int i = (int)(r % len[0]) + off[0];
    r /= len[0];
    int j = (int)(r % len[1]) + off[1];
    int k = (int)(r / len[1]) + off[2];
    const long long t = cell_index(bx, i, j, k);
    double gg = gchi[t] + carry[t], gr = gchi[bx.ntot + t] + carry[bx.ntot + t];
    carry[t] = 0.0;
    carry[bx.ntot + t] = 0.0;
    if (gg == 0.0 && gr == 0.0) continue;
    FlatCell<double> c[7];
    for (int m = 0; m < 7; ++m) {
      const long long cm = t + (m - 3) * st;
      c[m].pg = (p.gam - 1.0) * P[UU * bx.ntot + cm];
      c[m].pr = P[ER * bx.ntot + cm] * (1.0 / 3.0);
      c[m].vg = aux[(1 + 3 * d) * bx.ntot + cm];
      c[m].vr = aux[(2 + 3 * d) * bx.ntot + cm];
      c[m].w = aux[(3 + 3 * d) * bx.ntot + cm];
    }
    double Fg, Fr;
    flatten_cell<double>(c, &Fg, &Fr);
    const double pg_prev = prev ? prev[t] : 0.0, pr_prev = prev ? prev[bx.ntot + t] : 0.0;
    if (!(Fg > pg_prev)) {
      carry[t] = gg;
      gg = 0.0;
    }
    if (!(Fr > pr_prev)) {
      carry[bx.ntot + t] = gr;
      gr = 0.0;
    }
    if (gg == 0.0 && gr == 0.0) continue;
    for (int m = 0; m < 7; ++m) {
      FlatCell<D5> cd[7];
      for (int n = 0; n < 7; ++n) {
        const int o = n == m ? 0 : -100;
        cd[n].pg = D5::seed(c[n].pg, o);
        cd[n].pr = D5::seed(c[n].pr, o + 1);
        cd[n].vg = D5::seed(c[n].vg, o + 2);
        cd[n].vr = D5::seed(c[n].vr, o + 3);
        cd[n].w = D5::seed(c[n].w, o + 4);
      }
      D5 Fgd, Frd;
      flatten_cell<D5>(cd, &Fgd, &Frd);
      double v[5];
      for (int c5 = 0; c5 < 5; ++c5) v[c5] = gg * Fgd.d[c5] + gr * Frd.d[c5];
      const long long cm = t + (m - 3) * st;
      if (v[0] != 0.0) atomicAdd(&gP[UU * bx.ntot + cm], (p.gam - 1.0) * v[0]);
      if (v[1] != 0.0) atomicAdd(&gP[ER * bx.ntot + cm], v[1] * (1.0 / 3.0));
      if (v[2] != 0.0) atomicAdd(&gaux[cm], v[2]);
      if (v[3] != 0.0) atomicAdd(&gaux[bx.ntot + cm], v[3]);
      if (v[4] != 0.0) atomicAdd(&gaux[2 * bx.ntot + cm], v[4]);
    }
  }
}

// Cell factors of direction d (T): sqrt(-g) u^d, sqrt(-g) u^d_rad and
// w_d = min(1, 2 tau_d) of every cell.
template <int MET, int d>
__global__ void ka_prep(DevParams p, BoxGeo bx, const double* __restrict__ P, const double* __restrict__ K,
                        const double* __restrict__ gaux, double* gP, double* gk_out) {
  typedef Dn<3> D3;
  double gk = 0.0;
  for (long long t = HR_TID; t < bx.ntot; t += HR_STRIDE) {
    const double gvg = gaux[t], gvr = gaux[bx.ntot + t], gw = gaux[2 * bx.ntot + t];
    if (gvg == 0.0 && gvr == 0.0 && gw == 0.0) continue;
    long long r = t;
    const int i = (int)(r % bx.N[0]) - bx.ng[0];
    r /= bx.N[0];
    const int j = (int)(r % bx.N[1]) - bx.ng[1];
    const Geo<MET, D3> g = geo_cast<D3>(make_geo<MET, double>(p, xcen(bx, 0, i), xcen(bx, 1, j)));
    if (gvg != 0.0) {
      D3 ucon[4], ucov[4], gm;
      fourvel<MET, D3>(g, D3::seed(P[U1 * bx.ntot + t], 0), D3::seed(P[U2 * bx.ntot + t], 1),
                       D3::seed(P[U3 * bx.ntot + t], 2), ucon, ucov, &gm);
      const D3 v = g.gdet * ucon[d + 1];
      for (int c = 0; c < 3; ++c) gP[(U1 + c) * bx.ntot + t] += gvg * v.d[c];
    }
    if (gvr != 0.0) {
      D3 ucon[4], ucov[4], gm;
      fourvel<MET, D3>(g, D3::seed(P[UR1 * bx.ntot + t], 0), D3::seed(P[UR2 * bx.ntot + t], 1),
                       D3::seed(P[UR3 * bx.ntot + t], 2), ucon, ucov, &gm);
      const D3 v = g.gdet * ucon[d + 1];
      for (int c = 0; c < 3; ++c) gP[(UR1 + c) * bx.ntot + t] += gvr * v.d[c];
    }
    if (gw != 0.0) {
      D3 kabs, ksca;
      opacity<D3>(p, D3::seed(P[RHO * bx.ntot + t], 0), D3::seed(P[UU * bx.ntot + t], 1), D3(kfield(p, K, t)),
                  &kabs, &ksca, D3::seed(p.kscale, 2));
      const D3 tau = (kabs + ksca) * sqrt(g.gdd(d + 1)) * D3(bx.dx[d]);
      const D3 w = D3(2.0) * tau;
      if (w < 1.0) {
        gP[RHO * bx.ntot + t] += gw * w.d[0];
        gP[UU * bx.ntot + t] += gw * w.d[1];
        gk += gw * w.d[2];
      }
    }
  }
  warp_atomic_add(gk_out, gk);
}

// --------------------------------------------------------- ghost fill (T)
// Launched for d = 2, 1, 0 (the reverse of the forward order): every ghost
// cell's cotangent goes to its source cell, with the polar sign flips and the
// outflow clamps (derivative 1 where the clamp let the value through).
static __global__ void ka_bc_T(BoxGeo bx, const double* __restrict__ P, double* gP, int d) {
  int lo[3], len[3];
  for (int e = 0; e < 3; ++e) {
    if (e == d) {
      lo[e] = 0;
      len[e] = bx.ng[d];
    } else if (e < d) {
      lo[e] = -bx.ng[e];
      len[e] = bx.n[e] + 2 * bx.ng[e];
    } else {
      lo[e] = 0;
      len[e] = bx.n[e];
    }
  }
  const long long total = 2LL * len[0] * len[1] * len[2];
  for (long long id = HR_TID; id < total; id += HR_STRIDE) {
    long long r = id;
    int a0 = (int)(r % len[0]);
    r /= len[0];
    int a1 = (int)(r % len[1]);
    r /= len[1];
    int a2 = (int)(r % len[2]);
    int side = (int)(r / len[2]);
    int c[3] = {a0 + lo[0], a1 + lo[1], a2 + lo[2]};
    int g = c[d];
    int dst[3] = {c[0], c[1], c[2]}, src[3] = {c[0], c[1], c[2]};
    int bc = bx.bc[2 * d + side];
    dst[d] = side == 0 ? -1 - g : bx.n[d] + g;
    double sgn = 1.0;
    int clamp = 0;
    if (bc == 0) {
      src[d] = side == 0 ? bx.n[d] - 1 - g : g;
    } else if (bc == 1 || bc == 3) {
      src[d] = side == 0 ? 0 : bx.n[d] - 1;
      clamp = bc == 3 ? 0 : (side == 0 ? -1 : 1);
    } else {
      src[d] = side == 0 ? g : bx.n[d] - 1 - g;
      if (bx.n[2] > 1) src[2] = (c[2] + bx.n[2] / 2) % bx.n[2];
      sgn = -1.0;
    }
    const long long s = cell_index(bx, src[0], src[1], src[2]);
    const long long t = cell_index(bx, dst[0], dst[1], dst[2]);
    for (int q = 0; q < NPR; ++q) {
      double gv = gP[q * bx.ntot + t];
      gP[q * bx.ntot + t] = 0.0;
      if (gv == 0.0) continue;
      if (q == U1 + d || q == B1 + d || q == UR1 + d) gv *= sgn;
      if (clamp != 0 && (q == U1 + d || q == UR1 + d)) {
        const double v = P[q * bx.ntot + s] * sgn;
        if (clamp < 0 ? !(v < 0.0) : !(v > 0.0)) gv = 0.0;
      }
      if (gv != 0.0) atomicAdd(&gP[q * bx.ntot + s], gv);
    }
  }
}

// Active cells of gP -> gN (the cotangent of the previous sub-step's output).
static __global__ void ka_gather(BoxGeo bx, const double* __restrict__ gP, double* __restrict__ gN) {
  for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
    int i, j, k;
    zone_ijk(bx, z, i, j, k);
    const long long t = cell_index(bx, i, j, k);
    for (int q = 0; q < NPR; ++q) gN[q * bx.nact + z] = gP[q * bx.ntot + t];
  }
}

}  // namespace hr
