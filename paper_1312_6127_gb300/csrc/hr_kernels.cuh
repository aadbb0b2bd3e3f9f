// Kernels of one RK3 sub-step (Sec. 4.2 of McKinney et al. 2014) for sm_103a.
//
// Data layout in HBM: structure of arrays, one FP64 plane per primitive,
// [12][N3][N2][N1] with 4 ghost zones on each side of every active direction
// (i fastest, so a warp reads 32 consecutive x1 zones of one variable).
// Face fluxes of direction d share the cell indexing: the flux stored at cell
// t is the flux through t's lower d-face.
//
// A context holds one or more grids (the boxes of a batch).  Every array is
// the concatenation of per-grid blocks, each laid out as above; BoxGeo gives a
// grid's sizes and its offsets.  Every kernel loops over the grids and, inside
// a grid, over its index space with a grid-stride loop, so one launch advances
// all grids of a batch.  Grids are sized by the host in multiples of the SM
// count.
#pragma once
#include "hr_common.cuh"
#include "hr_implicit.cuh"

namespace hr {

struct Bufs {
  double* P;       // [12][ntot] primitives, ghosts included (per grid)
  double* K;       // [ntot] per-zone absorption opacity (opacity field mode), ghosts included
  double* Un;      // [12][nact] conserved state at the start of the step
  double* Sn;      // [nact] conserved entropy at the start of the step (RK3; null otherwise)
  void* F[3];      // [12][ntot] face fluxes (real type of the precision mode)
  void* FS[3];     // [ntot] entropy face fluxes (RK3; null otherwise)
  void* spd[3];    // [ntot] per-face max signal speed
  void* aux;       // [10][ntot] per-cell gdet, sqrt(-g) u^d gas/rad, tau weights
  void* flat[3];   // [2][ntot] flattener, max over the sub-steps of the step
  void* emf;       // [ntot] edge EMF scratch
  void* edges;     // [24][ntot] reconstructed edges of one direction
  double* dt;      // [nbox] time step of each grid
  unsigned char* status;  // [nact] worst outcome over the sub-steps
  int* iters;             // [nact] Newton steps summed over the sub-steps
  unsigned char* failed;  // [nact] back-up flag of the current sub-step
  int* qcount;            // [4] retry queue, back-up list, Newton continuation queue lengths
  int* qzone;             // [nact] retry queue: zone index within its grid
  int* qbox;              // [nact] retry queue: grid of the entry
  double* qdata;          // [nact][19] retry queue payload: U*, PMHD best x, e_T, h, S*
  int* fzone;             // [nact] back-up list: zone index within its grid
  int* fbox;              // [nact] back-up list: grid of the entry
  double* ftmp;           // [nact][12] averaged primitives of back-up zones
  int* czone;             // [nact] Newton continuation queue: zone index within its grid
  int* cbox;              // [nact] Newton continuation queue: grid of the entry
  double* cdata;          // [nact][CSTRIDE] continuation payload: U*, Newton state
  unsigned long long* stats;  // [8] counters
  unsigned long long* dtmin;  // [nbox] CFL minimum (ordered bits of a positive double)
  const double* geo;          // metric tables of Kerr-Schild grids (null otherwise)
  // records of the sub-step for the adjoint's recomputation of a step and for
  // the IMEX sources (null otherwise); planes per grid, grid b at 12 aoff_b:
  double* ust_rec;            // [12][nact] U* of every zone of the sub-step
  unsigned char* meth_rec;    // [nact] outcome of every zone of the sub-step
  double* psol_rec;           // [12][nact] solution of every zone before the floors
  double* sst_rec;            // [nact] explicit entropy S* of every zone of the sub-step
  double* imexM;              // IMEX: [4 stages][4 gas rows][nact] per grid, grid b at 16 aoff_b
  double* Bf[3];              // staggered field: sqrt(-g) B^d on the d-faces [ntot] (null: flux-CT)
};


// Counter update aggregated over the converged lanes of a warp.
__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned v) {
  unsigned mask = __activemask();
  unsigned s = __reduce_add_sync(mask, v);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && s) atomicAdd(dst, (unsigned long long)s);
}

#define HR_TID (blockIdx.x * (long long)blockDim.x + threadIdx.x)
#define HR_STRIDE ((long long)gridDim.x * blockDim.x)

// Opacity-field value of a cell (1 when the opacity is not a field).
__device__ __forceinline__ double kfield(const DevParams& p, const double* K, long long t) {
  return p.opacity == 2 ? K[t] : 1.0;
}

// ------------------------------------------------------------ metric tables
// The Kerr-Schild metric depends on (x1, x2) only.  A Kerr-Schild grid keeps,
// per (i, j), the metric at the cell centres, its x1 and x2 derivatives (for
// the geometric source) and the metric at the x1 and x2 faces, evaluated once
// when the context is created by the same functions the kernels would call.
// The FP64 kernels then read 16 doubles (L2-resident: a few MB per grid)
// instead of evaluating exp, sin, cos and four divisions per zone and face,
// which matters because the step is bound by FP64 arithmetic.
// Layout of a grid's table (offset BoxGeo::goff, in doubles): [16][N2][N1]
// centres, [16][N2][N1] centre derivatives, [16][N2][n1+1] x1 faces,
// [16][n2+1][N1] x2 faces; fields in the order of Geo (g00 g01 g03 g11 g13
// g22 g33 G00 G01 G11 G13 G22 G33 gdet alpha ialpha) and of MetricDeriv.
struct GeoTab {
  const double* C;
  const double* M;
  const double* F0;
  const double* F1;
  long long sC, sF0, sF1;  // plane sizes
};

__host__ __device__ __forceinline__ long long geotab_size(const BoxGeo& b) {
  const long long sC = (long long)b.N[0] * b.N[1];
  return 16 * (2 * sC + (long long)(b.n[0] + 1) * b.N[1] + (long long)b.N[0] * (b.n[1] + 1));
}

__device__ __forceinline__ GeoTab geotab(const double* base, const BoxGeo& b) {
  GeoTab t;
  t.sC = (long long)b.N[0] * b.N[1];
  t.sF0 = (long long)(b.n[0] + 1) * b.N[1];
  t.sF1 = (long long)b.N[0] * (b.n[1] + 1);
  t.C = base + b.goff;
  t.M = t.C + 16 * t.sC;
  t.F0 = t.M + 16 * t.sC;
  t.F1 = t.F0 + 16 * t.sF0;
  return t;
}

// entry of (i, j) (active indices, ghosts negative): centres, x1 faces
// (i = face index 0..n1), x2 faces (j = face index 0..n2)
__device__ __forceinline__ long long gidx_c(const BoxGeo& b, int i, int j) {
  return (long long)(j + b.ng[1]) * b.N[0] + (i + b.ng[0]);
}
__device__ __forceinline__ long long gidx_f0(const BoxGeo& b, int i, int j) {
  return (long long)(j + b.ng[1]) * (b.n[0] + 1) + i;
}
__device__ __forceinline__ long long gidx_f1(const BoxGeo& b, int i, int j) {
  return (long long)j * b.N[0] + (i + b.ng[0]);
}

template <int MET>
__device__ __forceinline__ Geo<MET, double> geo_load(const double* __restrict__ t, long long s, long long x) {
  Geo<MET, double> g;
  g.g00 = __ldg(t + x);
  g.g01 = __ldg(t + s + x);
  g.g03 = __ldg(t + 2 * s + x);
  g.g11 = __ldg(t + 3 * s + x);
  g.g13 = __ldg(t + 4 * s + x);
  g.g22 = __ldg(t + 5 * s + x);
  g.g33 = __ldg(t + 6 * s + x);
  g.G00 = __ldg(t + 7 * s + x);
  g.G01 = __ldg(t + 8 * s + x);
  g.G11 = __ldg(t + 9 * s + x);
  g.G13 = __ldg(t + 10 * s + x);
  g.G22 = __ldg(t + 11 * s + x);
  g.G33 = __ldg(t + 12 * s + x);
  g.gdet = __ldg(t + 13 * s + x);
  g.alpha = __ldg(t + 14 * s + x);
  g.ialpha = __ldg(t + 15 * s + x);
  return g;
}

template <int MET>
__device__ __forceinline__ void geo_store(double* t, long long s, long long x, const Geo<MET, double>& g) {
  const double v[16] = {g.g00, g.g01, g.g03, g.g11, g.g13, g.g22, g.g33, g.G00,
                        g.G01, g.G11, g.G13, g.G22, g.G33, g.gdet, g.alpha, g.ialpha};
  for (int f = 0; f < 16; ++f) t[f * s + x] = v[f];
}

// Metric of the centre of cell (i, j): from the table when the grid has one
// (FP64 kernels), else evaluated.
template <int MET, typename R>
__device__ __forceinline__ Geo<MET, R> geo_centre(const DevParams& p, const BoxGeo& bx, const double* geo0, int i,
                                                  int j) {
  if constexpr (MET == KS && std::is_same<R, double>::value) {
    if (geo0 && bx.goff >= 0) {
      const GeoTab T = geotab(geo0, bx);
      return geo_load<MET>(T.C, T.sC, gidx_c(bx, i, j));
    }
  }
  return make_geo<MET, R>(p, R(xcen(bx, 0, i)), R(xcen(bx, 1, j)));
}

// ----------------------------------------------------------- ghost fill
// One direction at a time, in the order 1, 2, 3, so that edges and corners
// come from already-filled cells.  Periodic wraps; outflow copies the last
// active zone and clamps the normal velocities (gas and radiation) so nothing
// enters from the ghost; polar mirrors across the axis from the zone half a
// turn away in phi, negating the theta components.  The opacity field, when
// present, is copied like a scalar primitive.
static __global__ void k_bc_fill(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                                 double* __restrict__ P0, double* __restrict__ K0, int d) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    double* P = P0 + 12 * bx.coff;
    double* K = K0 ? K0 + bx.coff : nullptr;
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
    long long total = 2LL * len[0] * len[1] * len[2];
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
      if (bc == 4) continue;  // fixed ghosts keep the values they were given
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
      long long s = cell_index(bx, src[0], src[1], src[2]);
      long long t = cell_index(bx, dst[0], dst[1], dst[2]);
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        double v = P[q * bx.ntot + s];
        if (q == U1 + d || q == B1 + d || q == UR1 + d) v *= sgn;
        if (clamp != 0 && (q == U1 + d || q == UR1 + d)) {
          const double vc = clamp < 0 ? fmin(v, 0.0) : fmax(v, 0.0);
          if (p.sig) sig_put(p, bx.coff + t, 50 + d, (unsigned long long)q << 8 | (vc != v ? 1u : 0u));
          v = vc;
        }
        P[q * bx.ntot + t] = v;
      }
      if (K) K[t] = K[s];
    }
  }
}

// --------------------------------------------------------------- cell prep
// Per cell: sqrt(-g), and for every active direction d the flattener inputs
// sqrt(-g) u^d (gas, radiation) and the weight w_d = min(1, 2 tau_d) of the
// optical depth of the cell along d (Sec. 4.3).
template <int MET, typename R>
__global__ void k_prep(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                       const double* __restrict__ P0, const double* __restrict__ K0,
                       R* __restrict__ aux0, const double* __restrict__ geo0) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    const double* K = K0 + bx.coff;
    R* aux = aux0 + 10 * bx.coff;
    for (long long t = HR_TID; t < bx.ntot; t += HR_STRIDE) {
      long long r = t;
      int i = (int)(r % bx.N[0]) - bx.ng[0];
      r /= bx.N[0];
      int j = (int)(r % bx.N[1]) - bx.ng[1];
      const Geo<MET, R> g = geo_centre<MET, R>(p, bx, geo0, i, j);
      R ucon[4], ucov[4], gm, urc[4], urv[4], gr;
      fourvel<MET, R>(g, R(P[U1 * bx.ntot + t]), R(P[U2 * bx.ntot + t]), R(P[U3 * bx.ntot + t]), ucon, ucov, &gm);
      fourvel<MET, R>(g, R(P[UR1 * bx.ntot + t]), R(P[UR2 * bx.ntot + t]), R(P[UR3 * bx.ntot + t]), urc, urv, &gr);
      R kabs, ksca;
      opacity<R>(p, R(P[RHO * bx.ntot + t]), R(P[UU * bx.ntot + t]), R(kfield(p, K, t)), &kabs, &ksca);
      aux[t] = g.gdet;
#pragma unroll
      for (int d = 1; d <= 3; ++d) {
        aux[(1 + 3 * (d - 1)) * bx.ntot + t] = g.gdet * ucon[d];
        aux[(2 + 3 * (d - 1)) * bx.ntot + t] = g.gdet * urc[d];
        R tau = (kabs + ksca) * sqrt(g.gdd(d)) * R(bx.dx[d - 1]);
        R w = R(2) * tau;
        aux[(3 + 3 * (d - 1)) * bx.ntot + t] = w < R(1) ? w : R(1);
      }
    }
  }
}

// ----------------------------------------------------------- flattener
// Shock flattener of Sec. 4.3 (SP0 = 0.75): for GAS (gas pressure and
// sqrt(-g) u^d) and RAD (radiation pressure and sqrt(-g) u^d_rad), each
// pressure blended toward the total by the cell's w; flattening where
// |dp| > 0.33 min p and the flow compresses, with the shock parameter
// dp1/dp2 mapped by 10 (Sp - 0.75) to [0, 1]; the upstream neighbour's value
// is max-ed in; GAS and RAD are blended to their maximum by w; and the result
// is max-ed with the values of the earlier sub-steps of the step.
template <typename R>
struct FlatCell {
  R pg, pr, vg, vr, w;
};

template <typename R>
__device__ __forceinline__ R ftilde(const FlatCell<R>* c, int m, bool gas, R w) {
  R pe1 = gas ? c[m + 1].pg + w * c[m + 1].pr : c[m + 1].pr + w * c[m + 1].pg;
  R pem = gas ? c[m - 1].pg + w * c[m - 1].pr : c[m - 1].pr + w * c[m - 1].pg;
  R pe2 = gas ? c[m + 2].pg + w * c[m + 2].pr : c[m + 2].pr + w * c[m + 2].pg;
  R pe2m = gas ? c[m - 2].pg + w * c[m - 2].pr : c[m - 2].pr + w * c[m - 2].pg;
  R dp1 = pe1 - pem, dp2 = pe2 - pe2m;
  R dv = gas ? c[m + 1].vg - c[m - 1].vg : c[m + 1].vr - c[m - 1].vr;
  R mn = pe1 < pem ? pe1 : pem;
  if (fabs(dp1) > R(0.33) * mn && dv < R(0)) {
    R sp = dp2 != R(0) ? dp1 / dp2 : R(0);
    R f = R(10) * (sp - R(0.75));
    return f < R(0) ? R(0) : (f > R(1) ? R(1) : f);
  }
  return R(0);
}

// Flattener of the centre cell c[3] of a 7-cell stencil (GAS, RAD).
template <typename R>
__device__ __forceinline__ void flatten_cell(const FlatCell<R>* c, R* Fg, R* Fr) {
  const R w = c[3].w;
  R g0 = ftilde<R>(c, 3, true, w), r0 = ftilde<R>(c, 3, false, w);
  R pg1 = c[4].pg + w * c[4].pr, pgm = c[2].pg + w * c[2].pr;
  R pr1 = c[4].pr + w * c[4].pg, prm = c[2].pr + w * c[2].pg;
  int sg = (pg1 - pgm) < R(0) ? 1 : -1;
  int sr = (pr1 - prm) < R(0) ? 1 : -1;
  R gn = ftilde<R>(c, 3 + sg, true, c[3 + sg].w);
  R rn = ftilde<R>(c, 3 + sr, false, c[3 + sr].w);
  R fg = g0 > gn ? g0 : gn;
  R fr = r0 > rn ? r0 : rn;
  R mx = fg > fr ? fg : fr;
  *Fg = (R(1) - w) * fg + w * mx;
  *Fr = (R(1) - w) * fr + w * mx;
}

// Branches of the flattener of cell 3 of c[0..6] (flatten_cell): each
// ftilde's compression test and clamp, the neighbour chosen, the maxima taken.
template <typename R>
__device__ __forceinline__ unsigned ftilde_code(const FlatCell<R>* c, int m, bool gas, R w) {
  auto pe = [&](int o) { return gas ? c[m + o].pg + w * c[m + o].pr : c[m + o].pr + w * c[m + o].pg; };
  auto ve = [&](int o) { return gas ? c[m + o].vg : c[m + o].vr; };
  R dp1 = pe(1) - pe(-1), dp2 = pe(2) - pe(-2);
  R dv = ve(1) - ve(-1);
  R p1 = pe(1), pm = pe(-1);
  if (!(fabs(dp1) > R(0.33) * (p1 < pm ? p1 : pm) && dv < R(0))) return 0u;
  R sp = dp2 != R(0) ? dp1 / dp2 : R(0);
  R f = R(10) * (sp - R(0.75));
  return f <= R(0) ? 1u : (f >= R(1) ? 3u : 2u);
}
template <typename R>
__device__ __forceinline__ unsigned flatten_code(const FlatCell<R>* c, R og, R orr) {
  const R w = c[3].w;
  R g0 = ftilde<R>(c, 3, true, w), r0 = ftilde<R>(c, 3, false, w);
  R pg1 = c[4].pg + w * c[4].pr, pgm = c[2].pg + w * c[2].pr;
  R pr1 = c[4].pr + w * c[4].pg, prm = c[2].pr + w * c[2].pg;
  int sg = (pg1 - pgm) < R(0) ? 1 : -1;
  int sr = (pr1 - prm) < R(0) ? 1 : -1;
  R gn = ftilde<R>(c, 3 + sg, true, c[3 + sg].w);
  R rn = ftilde<R>(c, 3 + sr, false, c[3 + sr].w);
  R fg = g0 > gn ? g0 : gn, fr = r0 > rn ? r0 : rn;
  R Fg = (R(1) - w) * fg + w * (fg > fr ? fg : fr), Fr = (R(1) - w) * fr + w * (fg > fr ? fg : fr);
  unsigned k = ftilde_code<R>(c, 3, true, w) | ftilde_code<R>(c, 3, false, w) << 2 |
               ftilde_code<R>(c, 3 + sg, true, c[3 + sg].w) << 4 | ftilde_code<R>(c, 3 + sr, false, c[3 + sr].w) << 6;
  k |= (sg > 0 ? 1u : 0u) << 8 | (sr > 0 ? 1u : 0u) << 9 | (g0 > gn ? 1u : 0u) << 10 | (r0 > rn ? 1u : 0u) << 11;
  k |= (fg > fr ? 1u : 0u) << 12 | (Fg > og ? 1u : 0u) << 13 | (Fr > orr ? 1u : 0u) << 14;
  return k;
}

template <typename R>
__global__ void k_flatten(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                          const double* __restrict__ P0, const R* __restrict__ aux0,
                          R* __restrict__ flat0, int d) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    const R* aux = aux0 + 10 * bx.coff;
    R* flat = flat0 + 2 * bx.coff;
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
    long long total = (long long)len[0] * len[1] * len[2];
    const long long st = bx.str[d];
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int i = (int)(r % len[0]) + off[0];
      r /= len[0];
      int j = (int)(r % len[1]) + off[1];
      int k = (int)(r / len[1]) + off[2];
      long long t = cell_index(bx, i, j, k);
      FlatCell<R> c[7];
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        long long cm = t + (m - 3) * st;
        c[m].pg = R((p.gam - 1.0) * P[UU * bx.ntot + cm]);
        c[m].pr = R(P[ER * bx.ntot + cm] * (1.0 / 3.0));
        c[m].vg = aux[(1 + 3 * d) * bx.ntot + cm];
        c[m].vr = aux[(2 + 3 * d) * bx.ntot + cm];
        c[m].w = aux[(3 + 3 * d) * bx.ntot + cm];
      }
      R Fg, Fr;
      flatten_cell<R>(c, &Fg, &Fr);
      R og = flat[t], orr = flat[bx.ntot + t];
      if (p.sig) sig_put(p, bx.coff + t, 30 + d, flatten_code<R>(c, og, orr));
      flat[t] = Fg > og ? Fg : og;
      flat[bx.ntot + t] = Fr > orr ? Fr : orr;
    }
  }
}

// ------------------------------------------------------------- reconstruction
template <typename R>
__device__ __forceinline__ R mc_slope(R qm, R q0, R qp) {
  R dl = q0 - qm, dr = qp - q0, dc = R(0.5) * (qp - qm);
  if (dl * dr <= R(0)) return R(0);
  R m = fabs(dc);
  R a = R(2) * fabs(dl), b = R(2) * fabs(dr);
  m = m < a ? m : a;
  m = m < b ? m : b;
  return dc > R(0) ? m : -m;
}

// Branch of mc_slope: 0 opposite one-sided slopes (zero), 1 central,
// 2 twice the left, 3 twice the right difference.
template <typename R>
__device__ __forceinline__ unsigned mc_code(R qm, R q0, R qp) {
  R dl = q0 - qm, dr = qp - q0, dc = R(0.5) * (qp - qm);
  if (dl * dr <= R(0)) return 0u;
  R m = fabs(dc);
  R a = R(2) * fabs(dl), b = R(2) * fabs(dr);
  unsigned c = 1u;
  if (a < m) {
    m = a;
    c = 2u;
  }
  if (b < m) c = 3u;
  return c;
}

// Branch of the PPM monotonicity limiter (ppm_slopes): 0 none, 1 flat,
// 2 left edge moved, 3 right edge moved.
template <typename R>
__device__ __forceinline__ unsigned ppm_code(R sm, R s0, R sp, R dm, R d0, R dp, R chi) {
  const R sixth = R(1.0 / 6.0);
  R l = R(0.5) * (sm + s0) - (d0 - dm) * sixth;
  R r = R(0.5) * (s0 + sp) - (dp - d0) * sixth;
  R q = s0;
  l = (R(1) - chi) * l + chi * q;
  r = (R(1) - chi) * r + chi * q;
  if ((r - q) * (q - l) <= R(0)) return 1u;
  R dd = r - l;
  R m6 = R(6) * (q - R(0.5) * (l + r));
  if (dd * m6 > dd * dd) return 2u;
  if (-dd * dd > dd * m6) return 3u;
  return 0u;
}

// PPM edge values of the centre of s[0..4] (Colella & Woodward 1984, no
// contact steepening), flattened toward the cell mean by chi, then limited.
// sm, s0, sp: the cell and its neighbours; dm, d0, dp: their MC slopes.
template <typename R>
__device__ __forceinline__ void ppm_slopes(R sm, R s0, R sp, R dm, R d0, R dp, R chi, R* aL, R* aR) {
  const R sixth = R(1.0 / 6.0);
  R l = R(0.5) * (sm + s0) - (d0 - dm) * sixth;
  R r = R(0.5) * (s0 + sp) - (dp - d0) * sixth;
  R q = s0;
  l = (R(1) - chi) * l + chi * q;
  r = (R(1) - chi) * r + chi * q;
  if ((r - q) * (q - l) <= R(0)) {
    l = q;
    r = q;
  } else {
    R dd = r - l;
    R m6 = R(6) * (q - R(0.5) * (l + r));
    if (dd * m6 > dd * dd) l = R(3) * q - R(2) * r;
    else if (-dd * dd > dd * m6) r = R(3) * q - R(2) * l;
  }
  *aL = l;
  *aR = r;
}

template <typename R>
__device__ __forceinline__ void ppm_cell(const R s[5], R chi, R* aL, R* aR) {
  R dm = mc_slope<R>(s[0], s[1], s[2]);
  R d0 = mc_slope<R>(s[1], s[2], s[3]);
  R dp = mc_slope<R>(s[2], s[3], s[4]);
  ppm_slopes<R>(s[1], s[2], s[3], dm, d0, dp, chi, aL, aR);
}

// ------------------------------------------------------- edge reconstruction
// MC slopes of all 12 primitives along d, once per cell: the PPM edges of a
// cell need the slopes of the cell and of its two neighbours, so computing
// them here saves two of every three slope evaluations of the edge kernel.
// Range: cells -2..n_d+1 along d, transverse range widened by one layer.  In
// r and phi on the Kerr-Schild grid the velocity and field components are
// reconstructed as sqrt(-g) times the primitive (Sec. 4.3).
template <int MET, typename R, int d>
__global__ void __launch_bounds__(256) k_slopes(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                                                const double* __restrict__ P0, const R* __restrict__ aux0,
                                                R* __restrict__ S0) {
  const bool weighted = (MET == KS) && (d != 1);
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    const R* aux = aux0 + 10 * bx.coff;
    R* S = S0 + 12 * bx.coff;
    int len[3], off[3];
    for (int e = 0; e < 3; ++e) {
      if (bx.n[e] > 1) {
        len[e] = bx.n[e] + (e == d ? 4 : 2);
        off[e] = e == d ? -2 : -1;
      } else {
        len[e] = 1;
        off[e] = 0;
      }
    }
    long long total = (long long)len[0] * len[1] * len[2];
    const long long st = bx.str[d];
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int i = (int)(r % len[0]) + off[0];
      r /= len[0];
      int j = (int)(r % len[1]) + off[1];
      int k = (int)(r / len[1]) + off[2];
      long long t = cell_index(bx, i, j, k);
      R gw[3];
      if (weighted) {
#pragma unroll
        for (int m = 0; m < 3; ++m) gw[m] = aux[t + (m - 1) * st];
      }
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
        R s[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          R v = R(P[q * bx.ntot + t + (m - 1) * st]);
          s[m] = wq ? gw[m] * v : v;
        }
        S[q * bx.ntot + t] = mc_slope<R>(s[0], s[1], s[2]);
        if (p.sig) sig_put(p, bx.coff + t, 10 + d, (unsigned long long)q << 8 | mc_code<R>(s[0], s[1], s[2]));
      }
    }
  }
}

// One thread per cell of the face range of direction d (cells -1..n_d along d,
// transverse range widened by one layer): the cell's PPM parabola (or MC
// slope) for all 12 primitives from the slopes of k_slopes (S0; null: the
// slopes are computed here, as the FP32 path does), flattened by the
// cell's GAS or RAD flattener, stored as the two edge values E[0][q] (lower)
// and E[1][q] (upper).  Every parabola is built once per direction; the face
// kernel reads the upper edge of cell f-1 and the lower edge of cell f.
template <int MET, typename R, int d>
__global__ void __launch_bounds__(256) k_edges(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                                               const double* __restrict__ P0, const R* __restrict__ aux0,
                                               const R* __restrict__ flat0, const R* __restrict__ S0,
                                               R* __restrict__ E0) {
  const bool weighted = (MET == KS) && (d != 1);
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    const R* aux = aux0 + 10 * bx.coff;
    const R* flat = flat0 + 2 * bx.coff;
    const R* S = S0 + 12 * bx.coff;
    R* E = E0 + 24 * bx.coff;
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
    long long total = (long long)len[0] * len[1] * len[2];
    const long long st = bx.str[d];
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int i = (int)(r % len[0]) + off[0];
      r /= len[0];
      int j = (int)(r % len[1]) + off[1];
      int k = (int)(r / len[1]) + off[2];
      long long t = cell_index(bx, i, j, k);
      R chg = R(0), chr = R(0);
      if (p.recon == 0) {
        chg = flat[t];
        chr = flat[bx.ntot + t];
      }
      if (!S0) {  // slopes computed here (FP32, where arithmetic is cheap)
        R gw[5];
        if (weighted) {
#pragma unroll
          for (int m = 0; m < 5; ++m) gw[m] = aux[t + (m - 2) * st];
        }
#pragma unroll
        for (int q = 0; q < NPR; ++q) {
          const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
          R s[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            R v = R(P[q * bx.ntot + t + (m - 2) * st]);
            s[m] = wq ? gw[m] * v : v;
          }
          R aL, aR;
          if (p.recon == 0) {
            ppm_cell<R>(s, q < ER ? chg : chr, &aL, &aR);
          } else {
            R dq = mc_slope<R>(s[1], s[2], s[3]);
            aL = s[2] - R(0.5) * dq;
            aR = s[2] + R(0.5) * dq;
          }
          E[q * bx.ntot + t] = aL;
          E[(NPR + q) * bx.ntot + t] = aR;
        }
        continue;
      }
      R gw[3];
      if (weighted && p.recon == 0) {
#pragma unroll
        for (int m = 0; m < 3; ++m) gw[m] = aux[t + (m - 1) * st];
      }
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
        R aL, aR;
        if (p.recon == 0) {
          R s[3], ds[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            R v = R(P[q * bx.ntot + t + (m - 1) * st]);
            s[m] = wq ? gw[m] * v : v;
            ds[m] = S[q * bx.ntot + t + (m - 1) * st];
          }
          ppm_slopes<R>(s[0], s[1], s[2], ds[0], ds[1], ds[2], q < ER ? chg : chr, &aL, &aR);
          if (p.sig)
            sig_put(p, bx.coff + t, 20 + d,
                    (unsigned long long)q << 8 | ppm_code<R>(s[0], s[1], s[2], ds[0], ds[1], ds[2], q < ER ? chg : chr));
        } else {
          R v = R(P[q * bx.ntot + t]);
          if (wq) v = aux[t] * v;
          const R dq = S[q * bx.ntot + t];
          aL = v - R(0.5) * dq;
          aR = v + R(0.5) * dq;
        }
        E[q * bx.ntot + t] = aL;
        E[(NPR + q) * bx.ntot + t] = aR;
      }
    }
  }
}

// Riemann flux through one face of direction d (0-based) from the two
// reconstructed states: both states' gas and radiation signal speeds, then
// HLL or LAXF (Eqs. hll, lax), the gas and radiation groups with their own
// speeds; F[B_d] = 0.  smax: the largest signal speed (for the CFL step).
// Used by the face kernel and, on dual numbers, by the adjoint.
template <int MET, typename R, int d>
__device__ __forceinline__ void face_flux(const DevParams& p, const Geo<MET, R>& g, R dxd, R kL, R kR, R ks,
                                          const R PL[NPR], const R PR[NPR], R out[NPR], R* smax,
                                          unsigned* code = nullptr, R* fs = nullptr, R* gas = nullptr) {
  R sL[4], sR[4];
  unsigned cL = 0, cR = 0;
  R lL[3], lR[3];  // Lorentz factors and 1/u^t of the states, for face_accum
  const R dl = sqrt(g.gdd(d + 1)) * dxd;  // proper cell length along d, for the optical depth
  face_speeds<MET, R>(p, g, d + 1, dl, kL, ks, PL, sL, code ? &cL : nullptr, lL);
  face_speeds<MET, R>(p, g, d + 1, dl, kR, ks, PR, sR, code ? &cR : nullptr, lR);
  R cmaxg = fmax(R(0), fmax(sL[1], sR[1]));
  R cming = -fmin(R(0), fmin(sL[0], sR[0]));
  R cmaxr = fmax(R(0), fmax(sL[3], sR[3]));
  R cminr = -fmin(R(0), fmin(sL[2], sR[2]));
  if (code) {  // which signal speed each maximum took, and the speed caps
    unsigned c = cL | (cR << 3);
    c |= (sL[1] >= sR[1] ? 0u : 1u) << 6 | (R(0) > fmax(sL[1], sR[1]) ? 1u : 0u) << 7;
    c |= (sL[0] <= sR[0] ? 0u : 1u) << 8 | (R(0) < fmin(sL[0], sR[0]) ? 1u : 0u) << 9;
    c |= (sL[3] >= sR[3] ? 0u : 1u) << 10 | (R(0) > fmax(sL[3], sR[3]) ? 1u : 0u) << 11;
    c |= (sL[2] <= sR[2] ? 0u : 1u) << 12 | (R(0) < fmin(sL[2], sR[2]) ? 1u : 0u) << 13;
    c |= (cmaxg > cming ? 1u : 0u) << 14 | (cmaxr > cminr ? 1u : 0u) << 15;
    *code = c;
  }
  // weights of (F_L, U_L) and (F_R, U_R) in the flux, gas and radiation groups
  R fLg, uLg, fRg, uRg, fLr, uLr, fRr, uRr;
  if (p.flux == 0) {  // LAXF: 1/2 (F_L + F_R - c (U_R - U_L))
    R cg = cmaxg > cming ? cmaxg : cming, cr = cmaxr > cminr ? cmaxr : cminr;
    fLg = fRg = fLr = fRr = R(0.5);
    uLg = R(0.5) * cg;
    uRg = -uLg;
    uLr = R(0.5) * cr;
    uRr = -uLr;
  } else {  // HLL: (c- F_R + c+ F_L - c- c+ (U_R - U_L)) / (c- + c+)
    R sg = cmaxg + cming, sr = cmaxr + cminr;
    if (sg > R(0)) {
      R isg = R(1) / sg;
      fLg = cmaxg * isg;
      fRg = cming * isg;
      uLg = cming * cmaxg * isg;
      uRg = -uLg;
    } else {
      fLg = fRg = R(0.5);
      uLg = uRg = R(0);
    }
    if (sr > R(0)) {
      R isr = R(1) / sr;
      fLr = cmaxr * isr;
      fRr = cminr * isr;
      uLr = cminr * cmaxr * isr;
      uRr = -uLr;
    } else {
      fLr = fRr = R(0.5);
      uLr = uRr = R(0);
    }
  }
#pragma unroll
  for (int q = 0; q < NPR; ++q) out[q] = R(0);
  if (fs) *fs = R(0);
  face_accum<MET, R>(p, g, d + 1, PL, fLg, uLg, fLr, uLr, out, fs, lL);
  face_accum<MET, R>(p, g, d + 1, PR, fRg, uRg, fRr, uRr, out, fs, lR);
  out[B1 + d] = R(0);
  *smax = fmax(fmax(cmaxg, cming), fmax(cmaxr, cminr));
  if (gas) {
    gas[0] = cmaxg;
    gas[1] = cming;
  }
}

// ----------------------------------------------------------------- fluxes
// One thread per face of direction d (faces 0..n_d, transverse range widened
// by one layer for the EMF averages).  Reads the two reconstructed states
// (upper edge of cell f-1, lower edge of cell f), evaluates the metric at the
// face in registers, the gas and radiation signal speeds of both states and
// the HLL or LAXF flux (Eqs. hll, lax), gas and radiation groups with their own
// speeds.  The direction is a template parameter so that every index into a
// 4-vector or the primitive array is resolved at compile time.
template <int MET, typename R, int d>
__global__ void __launch_bounds__(128) k_face(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                                              const R* __restrict__ E0, const double* __restrict__ K0,
                                              R* __restrict__ F0, R* __restrict__ spd0,
                                              const double* __restrict__ geo0, R* __restrict__ FS0,
                                              R* __restrict__ gsp0 = nullptr) {
  const bool weighted = (MET == KS) && (d != 1);
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const R* E = E0 + 24 * bx.coff;
    const double* K = K0 + bx.coff;
    R* F = F0 + 12 * bx.coff;
    R* spd = spd0 + bx.coff;
    R* FS = FS0 ? FS0 + bx.coff : nullptr;
    R* gsp = gsp0 ? gsp0 + 2 * bx.coff : nullptr;  // gas v_max, v_min per face (staggered field)
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
    long long total = (long long)len[0] * len[1] * len[2];
    const long long st = bx.str[d];
    const R dxd = R(bx.dx[d]);
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int ii[3];
      ii[0] = (int)(r % len[0]) + off[0];
      r /= len[0];
      ii[1] = (int)(r % len[1]) + off[1];
      ii[2] = (int)(r / len[1]) + off[2];
      long long t = cell_index(bx, ii[0], ii[1], ii[2]);
      const int f = ii[d];
      if (MET == KS && d == 1 && ((f == 0 && bx.bc[2] == 2) || (f == bx.n[1] && bx.bc[3] == 2))) {
#pragma unroll
        for (int q = 0; q < NPR; ++q) F[q * bx.ntot + t] = R(0);
        spd[t] = R(0);
        if (FS) FS[t] = R(0);
        if (gsp) gsp[t] = gsp[bx.ntot + t] = R(0);
        continue;
      }
      Geo<MET, R> g;
      bool tab = false;
      if constexpr (MET == KS && std::is_same<R, double>::value) {
        if (geo0 && bx.goff >= 0) {
          const GeoTab T = geotab(geo0, bx);
          if (d == 0) g = geo_load<MET>(T.F0, T.sF0, gidx_f0(bx, ii[0], ii[1]));
          else if (d == 1) g = geo_load<MET>(T.F1, T.sF1, gidx_f1(bx, ii[0], ii[1]));
          else g = geo_load<MET>(T.C, T.sC, gidx_c(bx, ii[0], ii[1]));
          tab = true;
        }
      }
      if (!tab) {
        R xf[3];
        for (int e = 0; e < 3; ++e) xf[e] = R(bx.x0[e] + (ii[e] + (e == d ? 0.0 : 0.5)) * bx.dx[e]);
        g = make_geo<MET, R>(p, xf[0], xf[1]);
      }
      const R igf = weighted ? R(1) / g.gdet : R(1);
      R PL[NPR], PR[NPR];
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        const bool wq = weighted && ((q >= U1 && q <= B3) || q >= UR1);
        R aR = E[(NPR + q) * bx.ntot + t - st];  // upper edge of cell f-1
        R bL = E[q * bx.ntot + t];               // lower edge of cell f
        PL[q] = wq ? aR * igf : aR;
        PR[q] = wq ? bL * igf : bL;
      }
      const R kL = R(kfield(p, K, t - st)), kR = R(kfield(p, K, t));
      R out[NPR], smax;
      unsigned fcode = 0;
      R fsv, gs[2];
      face_flux<MET, R, d>(p, g, dxd, kL, kR, R(p.kscale), PL, PR, out, &smax, p.sig ? &fcode : nullptr,
                           FS ? &fsv : nullptr, gs);
      if (p.sig) sig_put(p, bx.coff + t, 40 + d, fcode);
      if (FS) FS[t] = fsv;
      if (gsp) {
        gsp[t] = gs[0];
        gsp[bx.ntot + t] = gs[1];
      }
#pragma unroll
      for (int q = 0; q < NPR; ++q) F[q * bx.ntot + t] = out[q];
      spd[t] = smax;
    }
  }
}

// ----------------------------------------------------------------- flux-CT
// Toth (2000) constrained transport for the pair (a, b) of active directions:
// edge EMF = 1/4 (F_a[B_b] + F_a[B_b](b-1) - F_b[B_a] - F_b[B_a](a-1)), zero on
// the polar axis; then F_a[B_b] and F_b[B_a] become averages of the two
// adjacent edge EMFs (with opposite signs).
template <typename R>
__global__ void k_emf(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, const R* __restrict__ Fa0,
                      const R* __restrict__ Fb0, R* __restrict__ emf0, int a, int b) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const R* fab = Fa0 + 12 * bx.coff + (B1 + b) * bx.ntot;
    const R* fba = Fb0 + 12 * bx.coff + (B1 + a) * bx.ntot;
    R* emf = emf0 + bx.coff;
    int len[3];
    for (int e = 0; e < 3; ++e) len[e] = bx.n[e] + ((e == a || e == b) ? 1 : 0);
    long long total = (long long)len[0] * len[1] * len[2];
    const long long sa = bx.str[a], sb = bx.str[b];
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int ii[3];
      ii[0] = (int)(r % len[0]);
      r /= len[0];
      ii[1] = (int)(r % len[1]);
      ii[2] = (int)(r / len[1]);
      long long t = cell_index(bx, ii[0], ii[1], ii[2]);
      bool pole = p.metric == KS && (a == 1 || b == 1) &&
                  ((ii[1] == 0 && bx.bc[2] == 2) || (ii[1] == bx.n[1] && bx.bc[3] == 2));
      emf[t] = pole ? R(0) : R(0.25) * (fab[t] + fab[t - sb] - fba[t] - fba[t - sa]);
    }
  }
}

template <typename R>
__global__ void k_ct(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, const R* __restrict__ emf0,
                     R* __restrict__ Fa0, R* __restrict__ Fb0, int a, int b) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    R* fab = Fa0 + 12 * bx.coff + (B1 + b) * bx.ntot;
    R* fba = Fb0 + 12 * bx.coff + (B1 + a) * bx.ntot;
    const R* emf = emf0 + bx.coff;
    // two index spaces: a-faces (a in [0,n_a], b in [0,n_b)) then b-faces
    int la[3], lb[3];
    for (int e = 0; e < 3; ++e) {
      la[e] = bx.n[e] + (e == a ? 1 : 0);
      lb[e] = bx.n[e] + (e == b ? 1 : 0);
    }
    long long na = (long long)la[0] * la[1] * la[2];
    long long nb = (long long)lb[0] * lb[1] * lb[2];
    const long long sa = bx.str[a], sb = bx.str[b];
    for (long long id = HR_TID; id < na + nb; id += HR_STRIDE) {
      const int* L = id < na ? la : lb;
      long long r = id < na ? id : id - na;
      int i0 = (int)(r % L[0]);
      r /= L[0];
      int i1 = (int)(r % L[1]);
      int i2 = (int)(r / L[1]);
      long long t = cell_index(bx, i0, i1, i2);
      if (id < na) fab[t] = R(0.5) * (emf[t] + emf[t + sb]);
      else fba[t] = R(-0.5) * (emf[t] + emf[t + sa]);
    }
  }
}

// ----------------------------------------------------------------- floors
// Lorentz-factor caps, density and internal-energy floors f0 r^pow,
// magnetisation caps b^2/rho, b^2/u_g, u_g/rho, and Ebar > 0.
// ln r of the cell centre at x1 (0 on the Minkowski grid, where the floors
// take r = 1): x1 itself when r = e^x1 (R0 = 0).
template <int MET>
__device__ __forceinline__ double log_r(const DevParams& p, double x1) {
  if constexpr (MET == KS) return p.R0 == 0.0 ? x1 : log(p.R0 + exp(x1));
  else return 0.0;
}

template <int MET, typename T = double>
__device__ __forceinline__ void apply_floors(const DevParams& p, const Geo<MET, T>& g, double lr, T P[NPR],
                                             unsigned* code = nullptr) {
  T gm = sqrt(1.0 + g.sq3(P[U1], P[U2], P[U3]));
  if (code) {  // which floors act (the branch signature)
    *code = 0;
    const T gr0 = sqrt(1.0 + g.sq3(P[UR1], P[UR2], P[UR3]));
    if (gm > p.ggas_max) *code |= 1u;
    if (gr0 > p.grad_max) *code |= 2u;
  }
  if (gm > p.ggas_max) {
    T f = sqrt((p.ggas_max * p.ggas_max - 1.0) / (gm * gm - 1.0));
    P[U1] *= f;
    P[U2] *= f;
    P[U3] *= f;
  }
  T gr = sqrt(1.0 + g.sq3(P[UR1], P[UR2], P[UR3]));
  if (gr > p.grad_max) {
    T f = sqrt((p.grad_max * p.grad_max - 1.0) / (gr * gr - 1.0));
    P[UR1] *= f;
    P[UR2] *= f;
    P[UR3] *= f;
  }
  T ucon[4], ucov[4], bcon[4], bcov[4], bsq;
  fourvel<MET, T>(g, P[U1], P[U2], P[U3], ucon, ucov, &gm);
  bvec<MET, T>(g, ucon, ucov, P[B1], P[B2], P[B3], bcon, bcov, &bsq);
  // f0 r^pow as exp(pow ln r): the floor needs ln r only (x1 itself on the
  // Kerr-Schild grid with R0 = 0, where r = e^x1)
  T rfl = T(p.rf0 * (p.rfp == 0.0 ? 1.0 : exp(p.rfp * lr)));
  T ufl = T(p.uf0 * (p.ufp == 0.0 ? 1.0 : exp(p.ufp * lr)));
  if (code) {
    const T rb = bsq / p.bsq_rho_max, ub = bsq / p.bsq_u_max;
    const T rf = fmax(rfl, rb), uf = fmax(ufl, ub);
    const T u1 = fmax(P[UU], uf);
    *code |= (rb > rfl ? 4u : 0u) | (ub > ufl ? 8u : 0u) | (rf > P[RHO] ? 16u : 0u) | (uf > P[UU] ? 32u : 0u) |
             (u1 / p.u_rho_max > fmax(P[RHO], rf) ? 64u : 0u) | (!(P[ER] > 0.0) ? 128u : 0u);
  }
  rfl = fmax(rfl, bsq / p.bsq_rho_max);
  ufl = fmax(ufl, bsq / p.bsq_u_max);
  P[RHO] = fmax(P[RHO], rfl);
  P[UU] = fmax(P[UU], ufl);
  P[RHO] = fmax(P[RHO], P[UU] / p.u_rho_max);
  if (!(P[ER] > 0.0)) P[ER] = T(1e-150);
}

// Final primitives of an accepted PMHD iterate: gas from x, B fixed, radiation
// re-inverted with BASIC if the TYPE2 branch saw a negative energy (Sec. 4.10).
// Final primitives from the error function's state at x (pmhd_res), without
// evaluating it again: gas from x, B fixed, radiation re-inverted with BASIC
// if the TYPE2 branch saw a negative energy (Sec. 4.10).
template <int MET>
__device__ __forceinline__ void pmhd_final_state(const DevParams& p, const ImpSys<MET>& s, const double x[4],
                                                 const ImpState& st, double P[NPR]) {
  P[RHO] = st.rho;
  P[UU] = x[0];
  P[U1] = x[1];
  P[U2] = x[2];
  P[U3] = x[3];
  P[B1] = s.B[0];
  P[B2] = s.B[1];
  P[B3] = s.B[2];
  double Pr[4] = {st.Pr[0], st.Pr[1], st.Pr[2], st.Pr[3]};
  if (st.negE) rad_invert<MET, double>(p, s.g, st.Rt_pre, 0, Pr);
  P[ER] = Pr[0];
  P[UR1] = Pr[1];
  P[UR2] = Pr[2];
  P[UR3] = Pr[3];
}

template <int MET, typename T = double>
__device__ __forceinline__ void pmhd_final(const DevParams& p, const ImpSysT<MET, T>& s, const T x[4], T P[NPR],
                                           T* Eg = nullptr, unsigned* code = nullptr) {
  ImpResT<T> r;
  ImpStateT<T> stt;
  pmhd_res<MET, T>(p, s, x, r, &stt, false);
  if (code) {  // the TYPE2 limiter's branch at the solution (the branch signature)
    T Prt[4];
    int lim = 0;
    rad_invert<MET, T>(p, s.g, stt.Rt_pre, 2, Prt, &lim);
    *code = (unsigned)r.negE | (unsigned)lim << 1;
  }
  if (Eg)
    for (int k = 0; k < 4; ++k) Eg[k] = r.Eg[k];
  P[RHO] = stt.rho;
  P[UU] = x[0];
  P[U1] = x[1];
  P[U2] = x[2];
  P[U3] = x[3];
  P[B1] = s.B[0];
  P[B2] = s.B[1];
  P[B3] = s.B[2];
  T Pr[4] = {stt.Pr[0], stt.Pr[1], stt.Pr[2], stt.Pr[3]};
  if (r.negE) rad_invert<MET, T>(p, s.g, stt.Rt_pre, 0, Pr);
  P[ER] = Pr[0];
  P[UR1] = Pr[1];
  P[UR2] = Pr[2];
  P[UR3] = Pr[3];
}

// Optical depth of a cell along its longest active proper edge, from the
// primitives P (the tau < 2/3 guess rules of Sec. 4.10).
template <int MET>
__device__ __forceinline__ double zone_tau(const DevParams& p, const Geo<MET, double>& g, const double dx[3],
                                           const double P[NPR], double kf) {
  double kabs, ksca;
  opacity<double>(p, P[RHO], P[UU], kf, &kabs, &ksca);
  double dl = 0.0;
#pragma unroll
  for (int d = 1; d <= 3; ++d)
    if (p.act[d - 1]) dl = fmax(dl, sqrt(g.gdd(d)) * dx[d - 1]);
  return (kabs + ksca) * dl;
}

// The retry methods after PMHD (Sec. 4.10-4.11).  URAD from the PMHD iterate
// where its e_T < 1e-4, else from P_s; then PRAD if neither reached 1e-9,
// guessed from the better earlier solution where its e_T < 1e-4, else from
// the optically thin limit (the M1 inversion of R*, no source) where
// tau < 2/3, else from P_s.  The lowest-error solution wins (the earlier
// method on ties); its primitives before the floors go to Pn.  px / peT: the
// PMHD iterate and its error (inf if none).  Returns the outcome: ST_PMHD,
// ST_URAD (URAD or PRAD), or ST_BACKUP when no residual was finite or the
// best e_T exceeds 1e-7; *eT_out its error, *steps_out the Newton steps.
template <int MET>
__device__ int retry_sequence(const DevParams& p, const Geo<MET, double>& g, const ImpSys<MET>& s,
                              const double Ps[NPR], const double px[4], double peT, double tau, double Pn[NPR],
                              double* eT_out, int* steps_out, bool subdom = false, double Sst = NAN) {
  const bool pfin = isfinite(peT);
  double Pb[NPR];
  if (pfin) {  // the PMHD iterate as its error function left it (TYPE2 radiation)
    ImpRes rr;
    ImpState stt;
    pmhd_res<MET>(p, s, px, rr, &stt, false);
    Pb[RHO] = stt.rho;
    Pb[UU] = px[0];
    Pb[U1] = px[1];
    Pb[U2] = px[2];
    Pb[U3] = px[3];
    Pb[B1] = s.B[0];
    Pb[B2] = s.B[1];
    Pb[B3] = s.B[2];
    for (int q = 0; q < 4; ++q) Pb[ER + q] = stt.Pr[q];
  }
  const double* Pg = (pfin && peT < 1e-4) ? Pb : Ps;
  double urc[4], urv[4], gr;
  fourvel<MET, double>(g, Pg[UR1], Pg[UR2], Pg[UR3], urc, urv, &gr);
  const double e43 = (4.0 / 3.0) * Pg[ER];
  double xr[4];
  xr[0] = e43 * urc[0] * urv[0] + Pg[ER] * (1.0 / 3.0);
  for (int n = 1; n < 4; ++n) xr[n] = e43 * urc[0] * urv[n];
  double gas[5] = {Pg[RHO], Pg[UU], Pg[U1], Pg[U2], Pg[U3]};
  double ux[4], ugas[5], ueT;
  int steps = newton_urad<MET>(p, s, xr, gas, ux, ugas, &ueT);
  int best = pfin ? 0 : -1;
  double beT = pfin ? peT : HUGE_VAL;
  if (isfinite(ueT) && (best < 0 || ueT < beT)) {
    best = 1;
    beT = ueT;
  }
  double qx[4], qgas[5], qeT = HUGE_VAL;
  if (!(beT < 1e-9)) {
    double xq[4], gq[5];
    if (best >= 0 && beT < 1e-4) {
      if (best == 0) {
        for (int q = 0; q < 4; ++q) xq[q] = Pb[ER + q];
        for (int q = 0; q < 5; ++q) gq[q] = Pb[q];
      } else {
        rad_invert<MET>(p, g, ux, 2, xq);
        for (int q = 0; q < 5; ++q) gq[q] = ugas[q];
      }
    } else {
      if (tau < 2.0 / 3.0) {
        rad_invert<MET>(p, g, s.Rs, 2, xq);
      } else {
        for (int q = 0; q < 4; ++q) xq[q] = Ps[ER + q];
      }
      for (int q = 0; q < 5; ++q) gq[q] = Ps[q];
    }
    steps += newton_rad<MET, true>(p, s, xq, gq, qx, qgas, &qeT);
    if (isfinite(qeT) && (best < 0 || qeT < beT)) {
      best = 2;
      beT = qeT;
    }
  }
  double sx[4];
  if (subdom && !(beT < 1e-9)) {
    // staged PMHD (Sec. 4.10): guessed from the gas of the best earlier
    // solution if its e_T < 1e-4 (else P_s), u_g from the specific entropy
    // S* / (rho0 u^t)* at the density of P_s where S* is given
    const double* gsrc = Ps;
    if (best >= 0 && beT < 1e-4) gsrc = best == 0 ? Pb : (best == 1 ? ugas : qgas);
    double xs[4] = {gsrc[UU], gsrc[U1], gsrc[U2], gsrc[U3]};
    entropy_ug_guess(p, Sst, s.Dlab * g.gdet, Ps[RHO], xs);
    double seT;
    steps += newton_pmhd_staged<MET>(p, s, xs, sx, &seT);
    if (isfinite(seT) && (best < 0 || seT < beT)) {
      best = 3;
      beT = seT;
    }
  }
  // then the staged URAD and PRAD, each from the primitives of the
  // lowest-error solution so far if its e_T < 1e-4 (as its error function
  // formed them), else from P_s
  double tx[2][4], tgas[2][5];
#pragma unroll 1
  for (int pr = 0; pr < 2 && subdom && !(beT < 1e-9); ++pr) {
    double Pq[NPR];
    for (int q = 0; q < NPR; ++q) Pq[q] = Ps[q];
    if (best >= 0 && beT < 1e-4) {
      if (best == 0 || best == 3) {
        ImpRes rr;
        ImpState stt;
        const double* bx = best == 0 ? px : sx;
        pmhd_res<MET>(p, s, bx, rr, &stt, false);
        Pq[RHO] = stt.rho;
        for (int c = 0; c < 4; ++c) Pq[UU + c] = bx[c];
        for (int c = 0; c < 4; ++c) Pq[ER + c] = stt.Pr[c];
      } else if (best == 1 || best == 4) {
        const double* gg = best == 1 ? ugas : tgas[0];
        for (int c = 0; c < 5; ++c) Pq[c] = gg[c];
        rad_invert<MET>(p, g, best == 1 ? ux : tx[0], 2, Pq + ER);
      } else {
        const double* gg = best == 2 ? qgas : tgas[1];
        const double* xx = best == 2 ? qx : tx[1];
        for (int c = 0; c < 5; ++c) Pq[c] = gg[c];
        for (int c = 0; c < 4; ++c) Pq[ER + c] = xx[c];
      }
    }
    double gq[5] = {Pq[RHO], Pq[UU], Pq[U1], Pq[U2], Pq[U3]}, x4[4], reT;
    if (pr == 1) {
      for (int c = 0; c < 4; ++c) x4[c] = Pq[ER + c];
      steps += newton_rad_staged<MET, true>(p, s, x4, gq, tx[1], tgas[1], &reT);
    } else {
      double urc2[4], urv2[4], gr2;
      fourvel<MET, double>(g, Pq[UR1], Pq[UR2], Pq[UR3], urc2, urv2, &gr2);
      const double e43q = (4.0 / 3.0) * Pq[ER];
      x4[0] = e43q * urc2[0] * urv2[0] + Pq[ER] * (1.0 / 3.0);
      for (int c = 1; c < 4; ++c) x4[c] = e43q * urc2[0] * urv2[c];
      steps += newton_rad_staged<MET, false>(p, s, x4, gq, tx[0], tgas[0], &reT);
    }
    if (isfinite(reT) && (best < 0 || reT < beT)) {
      best = 4 + pr;
      beT = reT;
    }
  }
  int method = ST_URAD;
  if (best == 0) {
    pmhd_final<MET>(p, s, px, Pn);
    method = ST_PMHD;
  } else if (best == 1) {
    for (int q = 0; q < 5; ++q) Pn[q] = ugas[q];
    double Pr[4];
    if (rad_invert<MET>(p, g, ux, 2, Pr)) rad_invert<MET>(p, g, ux, 0, Pr);
    for (int q = 0; q < 4; ++q) Pn[ER + q] = Pr[q];
  } else if (best == 2) {
    for (int q = 0; q < 5; ++q) Pn[q] = qgas[q];
    for (int q = 0; q < 4; ++q) Pn[ER + q] = qx[q];
  } else if (best == 3) {
    pmhd_final<MET>(p, s, sx, Pn);
  } else if (best == 4) {
    for (int q = 0; q < 5; ++q) Pn[q] = tgas[0][q];
    double Pr[4];
    if (rad_invert<MET>(p, g, tx[0], 2, Pr)) rad_invert<MET>(p, g, tx[0], 0, Pr);
    for (int q = 0; q < 4; ++q) Pn[ER + q] = Pr[q];
  } else if (best == 5) {
    for (int q = 0; q < 5; ++q) Pn[q] = tgas[1][q];
    for (int q = 0; q < 4; ++q) Pn[ER + q] = tx[1][q];
  } else {
    for (int q = 0; q < NPR; ++q) Pn[q] = Ps[q];
    method = ST_BACKUP;
    beT = HUGE_VAL;
  }
  Pn[B1] = s.B[0];
  Pn[B2] = s.B[1];
  Pn[B3] = s.B[2];
  if (beT > 1e-7) method = ST_BACKUP;
  *eT_out = beT;
  *steps_out = steps;
  return method;
}

// Metric derivatives for the geometric source: forward-mode pair (d/dx1, d/dx2).
struct D2 {
  double v, a, b;
};
__device__ __forceinline__ D2 operator+(D2 x, D2 y) { return {x.v + y.v, x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ D2 operator-(D2 x, D2 y) { return {x.v - y.v, x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ D2 operator*(D2 x, D2 y) {
  return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b};
}
__device__ __forceinline__ D2 operator*(double c, D2 y) { return {c * y.v, c * y.a, c * y.b}; }
__device__ __forceinline__ D2 operator/(D2 x, D2 y) {
  double iy = 1.0 / y.v;
  double q = x.v * iy;
  return {q, (x.a - q * y.a) * iy, (x.b - q * y.b) * iy};
}

// d_nu g_{mu kappa} (nu = x1, x2) of the covariant Kerr-Schild metric in the
// internal chart and d_nu sqrt(-g).
struct MetricDeriv {
  double g00[2], g01[2], g03[2], g11[2], g13[2], g22[2], g33[2], sg[2];
};
__device__ __forceinline__ MetricDeriv ks_derivs(const DevParams& p, double x1, double x2) {
  const double a = p.a, hh = p.h, pi = 3.14159265358979323846;
  double ex = exp(x1);
  D2 r = {p.R0 + ex, ex, 0.0};
  double s2x, c2x;
  sincospi(2.0 * x2, &s2x, &c2x);
  D2 th = {pi * x2 + 0.5 * (1.0 - hh) * s2x, 0.0, pi + (1.0 - hh) * pi * c2x};
  double st, ct;
  sincos(th.v, &st, &ct);
  D2 sth = {st, 0.0, ct * th.b}, cth = {ct, 0.0, -st * th.b};
  D2 J1 = {ex, ex, 0.0};
  D2 J2 = {pi * (1.0 + (1.0 - hh) * c2x), 0.0, -2.0 * pi * pi * (1.0 - hh) * s2x};
  const double J3 = 2.0 * pi;
  D2 s2 = sth * sth;
  D2 S = r * r + (a * a) * (cth * cth);
  D2 tr = (2.0 * r) / S;
  D2 one = {1.0, 0.0, 0.0};
  D2 m00 = tr - one;
  D2 m01 = tr * J1;
  D2 m03 = (-a * J3) * (tr * s2);
  D2 m11 = (one + tr) * J1 * J1;
  D2 m13 = (-a * J3) * (s2 * (one + tr) * J1);
  D2 m22 = S * J2 * J2;
  D2 m33 = (J3 * J3) * (s2 * (S + (a * a) * (s2 * (one + tr))));
  D2 sg = J3 * (S * sth * J1 * J2);
  MetricDeriv md;
  md.g00[0] = m00.a; md.g00[1] = m00.b;
  md.g01[0] = m01.a; md.g01[1] = m01.b;
  md.g03[0] = m03.a; md.g03[1] = m03.b;
  md.g11[0] = m11.a; md.g11[1] = m11.b;
  md.g13[0] = m13.a; md.g13[1] = m13.b;
  md.g22[0] = m22.a; md.g22[1] = m22.b;
  md.g33[0] = m33.a; md.g33[1] = m33.b;
  md.sg[0] = sg.a; md.sg[1] = sg.b;
  return md;
}

// v^mu v^kappa d_nu g_{mu kappa}
template <typename T>
__device__ __forceinline__ T qform(const MetricDeriv& m, int n, const T v[4]) {
  return m.g00[n] * v[0] * v[0] + 2.0 * m.g01[n] * v[0] * v[1] + 2.0 * m.g03[n] * v[0] * v[3] +
         m.g11[n] * v[1] * v[1] + 2.0 * m.g13[n] * v[1] * v[3] + m.g22[n] * v[2] * v[2] +
         m.g33[n] * v[3] * v[3];
}

__device__ __forceinline__ MetricDeriv md_load(const double* __restrict__ t, long long s, long long x) {
  MetricDeriv m;
  double* v = reinterpret_cast<double*>(&m);  // the 16 doubles of MetricDeriv, in declaration order
  for (int f = 0; f < 16; ++f) v[f] = __ldg(t + f * s + x);
  return m;
}

// Fills the metric tables of the Kerr-Schild grids of a context.
static __global__ void k_geo_init(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, double* geo0) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    if (bx.goff < 0) continue;
    const GeoTab T = geotab(geo0, bx);
    double* C = const_cast<double*>(T.C);
    double* M = const_cast<double*>(T.M);
    double* F0 = const_cast<double*>(T.F0);
    double* F1 = const_cast<double*>(T.F1);
    const long long total = 2 * T.sC + T.sF0 + T.sF1;
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      if (id < T.sC) {  // centres and their derivatives
        const int i = (int)(id % bx.N[0]) - bx.ng[0], j = (int)(id / bx.N[0]) - bx.ng[1];
        const double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
        geo_store<KS>(C, T.sC, id, make_geo<KS, double>(p, x1, x2));
        const MetricDeriv md = ks_derivs(p, x1, x2);
        const double* v = reinterpret_cast<const double*>(&md);
        for (int f = 0; f < 16; ++f) M[f * T.sC + id] = v[f];
      } else if (id < T.sC + T.sF0) {  // x1 faces
        const long long e = id - T.sC;
        const int i = (int)(e % (bx.n[0] + 1)), j = (int)(e / (bx.n[0] + 1)) - bx.ng[1];
        const double x1 = bx.x0[0] + (i + 0.0) * bx.dx[0], x2 = bx.x0[1] + (j + 0.5) * bx.dx[1];
        geo_store<KS>(F0, T.sF0, e, make_geo<KS, double>(p, x1, x2));
      } else if (id < T.sC + T.sF0 + T.sF1) {  // x2 faces
        const long long e = id - T.sC - T.sF0;
        const int i = (int)(e % bx.N[0]) - bx.ng[0], j = (int)(e / bx.N[0]);
        const double x1 = bx.x0[0] + (i + 0.5) * bx.dx[0], x2 = bx.x0[1] + (j + 0.0) * bx.dx[1];
        geo_store<KS>(F1, T.sF1, e, make_geo<KS, double>(p, x1, x2));
      }
    }
  }
}

// U(P) and the geometric source SM(P) of one zone (X = SM on return):
// SM_nu = 1/2 sqrt(-g) T^{mu kappa} d_nu g_{mu kappa}, equal to
// sqrt(-g) T^kappa_lambda Gamma^lambda_{nu kappa} for a symmetric T and nonzero
// only for nu = x1, x2 on the stationary axisymmetric metric.
template <int MET, typename T>
__device__ __forceinline__ void cons_source(const DevParams& p, const Geo<MET, T>& g, double x1, double x2,
                                            const T Ps[NPR], T Us[NPR], T X[NPR],
                                            const MetricDeriv* mdp = nullptr) {
  T ucon[4], ucov[4], gm, bcon[4], bcov[4], bsq, urc[4], urv[4], gr;
  fourvel<MET, T>(g, Ps[U1], Ps[U2], Ps[U3], ucon, ucov, &gm);
  bvec<MET, T>(g, ucon, ucov, Ps[B1], Ps[B2], Ps[B3], bcon, bcov, &bsq);
  fourvel<MET, T>(g, Ps[UR1], Ps[UR2], Ps[UR3], urc, urv, &gr);
  const T pg = (p.gam - 1.0) * Ps[UU];
  const T wb = Ps[RHO] + Ps[UU] + pg + bsq, pt = pg + 0.5 * bsq;
  const T gd = g.gdet, mt = Ps[RHO] * ucon[0];
  const T E = Ps[ER], e43 = (4.0 / 3.0) * E;
  Us[0] = gd * mt;
  Us[1] = gd * (wb * ucon[0] * ucov[0] + pt - bcon[0] * bcov[0] + mt);
#pragma unroll
  for (int n = 1; n < 4; ++n) Us[1 + n] = gd * (wb * ucon[0] * ucov[n] - bcon[0] * bcov[n]);
  Us[5] = gd * Ps[B1];
  Us[6] = gd * Ps[B2];
  Us[7] = gd * Ps[B3];
  Us[8] = gd * (e43 * urc[0] * urv[0] + E * (1.0 / 3.0));
#pragma unroll
  for (int n = 1; n < 4; ++n) Us[8 + n] = gd * (e43 * urc[0] * urv[n]);
#pragma unroll
  for (int q = 0; q < NPR; ++q) X[q] = T(0.0);
  if constexpr (MET == KS) {
    const MetricDeriv md = mdp ? *mdp : ks_derivs(p, x1, x2);
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      T qu = qform(md, n, ucon), qb = qform(md, n, bcon), qr = qform(md, n, urc);
      X[2 + n] = 0.5 * gd * (wb * qu - qb) + pt * md.sg[n];
      X[9 + n] = 0.5 * gd * e43 * qr + E * (1.0 / 3.0) * md.sg[n];
    }
  }
  (void)x1;
  (void)x2;
}

constexpr int CSTRIDE = NPR + 23;  // continuation queue record: U*, Newton state, S*

__device__ __forceinline__ void newton_state_store(const NewtonState& st, double* d) {
  for (int i = 0; i < 4; ++i) {
    d[i] = st.x[i];
    d[4 + i] = st.best_x[i];
  }
  d[8] = st.best_eT;
  d[9] = st.hs.t1;
  d[10] = st.hs.t2;
  d[11] = st.hs.t3;
  d[12] = st.hs.t4;
  d[13] = st.hs.i1;
  d[14] = st.hs.i2;
  d[15] = st.hs.i3;
  d[16] = st.hs.i4;
  d[17] = st.eps;
  d[18] = (double)st.hs.rises;
  d[19] = (double)st.k;
  d[20] = (double)st.steps;
  d[21] = (double)st.jac32;
}

__device__ __forceinline__ void newton_state_load(const double* d, NewtonState& st) {
  for (int i = 0; i < 4; ++i) {
    st.x[i] = d[i];
    st.best_x[i] = d[4 + i];
  }
  st.best_eT = d[8];
  st.hs.t1 = d[9];
  st.hs.t2 = d[10];
  st.hs.t3 = d[11];
  st.hs.t4 = d[12];
  st.hs.i1 = d[13];
  st.hs.i2 = d[14];
  st.hs.i3 = d[15];
  st.hs.i4 = d[16];
  st.eps = d[17];
  st.hs.rises = (int)d[18];
  st.k = (int)d[19];
  st.steps = (int)d[20];
  st.jac32 = (int)d[21];
}

// End of a zone's PMHD solve: accept (e_T < 1e-9: final primitives, floors,
// write) or queue the zone for URAD.  Returns whether it was accepted.
template <int MET>
__device__ __forceinline__ bool pmhd_finish(const DevParams& p, const BoxGeo& bx, int bi, long long z, long long t,
                                            double x1, const Geo<MET, double>& g, const ImpSys<MET>& s,
                                            const double Ust[NPR], double h, const double best_x[4],
                                            double beT, int steps, double* P, const Bufs& b, double Sst,
                                            double acc_tol = 1e-9, const ImpState* bst = nullptr) {
  const long long zg = bx.aoff + z;
  b.iters[zg] += steps;
  const bool accept = beT >= 0.0 && beT < acc_tol;  // beT < 0: sub-dominant radiation, URAD first
  if (accept) {
    double Pn[NPR];
    unsigned lcode = 0;
    if (bst && !p.sig)  // the state the Newton loop kept for its best iterate
      pmhd_final_state<MET>(p, s, best_x, *bst, Pn);
    else
      pmhd_final<MET, double>(p, s, best_x, Pn, nullptr, p.sig ? &lcode : nullptr);
    if (b.psol_rec)
      for (int q = 0; q < NPR; ++q) b.psol_rec[12 * bx.aoff + q * bx.nact + z] = Pn[q];
    unsigned fcode = 0;
    apply_floors<MET>(p, g, log_r<MET>(p, x1), Pn, p.sig ? &fcode : nullptr);
    if (p.sig) sig_put(p, bx.coff + t, 60, (fcode << 2 | lcode) << 4 | ST_PMHD);
#pragma unroll
    for (int q = 0; q < NPR; ++q) P[q * bx.ntot + t] = Pn[q];
    if (b.meth_rec) b.meth_rec[zg] = ST_PMHD;
  } else {
    int slot = atomicAdd(&b.qcount[0], 1);
    b.qzone[slot] = (int)z;
    b.qbox[slot] = bi;
    double* qd = b.qdata + (long long)slot * QSTRIDE;
#pragma unroll
    for (int q = 0; q < NPR; ++q) qd[q] = Ust[q];
    for (int q = 0; q < 4; ++q) qd[12 + q] = isfinite(beT) ? best_x[q] : 0.0;
    qd[16] = beT;
    qd[17] = h;
    qd[18] = Sst;
  }
  return accept;
}

// The radiation of a zone is "extremely sub-dominant" (Sec. 4.10) when its
// conserved energy in U* or its fluid-frame energy density
// Ehat = Ebar (4/3 gamma_rel^2 - 1/3) is below 10 eps_m of the gas's (u_g for
// Ehat).  PMHD recovers the radiation from the gas's round-off there, so such
// zones start with URAD.  (The relative change of the energy row over the
// explicit update, which the paper also lists, would flag every zone whose
// radiation the update left unchanged, whatever its size; it is not used.)
template <int MET>
__device__ __forceinline__ bool radiation_subdominant(const Geo<MET, double>& g, const double Ust[NPR],
                                                      const double Ps[NPR]) {
  const double tiny = 10.0 * 2.220446049250313e-16;
  if (fabs(Ust[ER]) < tiny * fabs(Ust[UU])) return true;
  if (!(Ps[ER] < tiny * Ps[UU])) return false;  // Ehat >= Ebar (gamma_rel >= 1)
  double uc[4], uv[4], gm, rc[4], rv[4], gr;
  fourvel<MET, double>(g, Ps[U1], Ps[U2], Ps[U3], uc, uv, &gm);
  fourvel<MET, double>(g, Ps[UR1], Ps[UR2], Ps[UR3], rc, rv, &gr);
  const double grel = -(rc[0] * uv[0] + rc[1] * uv[1] + rc[2] * uv[2] + rc[3] * uv[3]);
  return Ps[ER] * ((4.0 / 3.0) * grel * grel - 1.0 / 3.0) < tiny * Ps[UU];
}

// Sec. 4.11: the cold-MHD equations are tried only for a cold, momentum-
// dominated zone: u_g < 0.1 rho0 u~^i u~_i of the guess primitives, and for
// the gas t^t_mu = T^t_mu + rho0 u^t delta^t_mu and the radiation R^t_mu of
// U* alike, |t_t t^t| < 0.1 |sum_i t_i t^i| with t^mu = g^{mu nu} t_nu.
template <int MET>
__device__ __forceinline__ bool cold_allowed(const Geo<MET, double>& g, const double Ust[NPR],
                                             const double Ps[NPR]) {
  if (!(Ps[UU] < 0.1 * Ps[RHO] * g.sq3(Ps[U1], Ps[U2], Ps[U3]))) return false;
  const double igd = 1.0 / g.gdet;
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    const int o = w == 0 ? UU : ER;
    const double t[4] = {Ust[o] * igd, Ust[o + 1] * igd, Ust[o + 2] * igd, Ust[o + 3] * igd};
    double up[3];
    g.raise3(t, up);
    const double at = fabs(t[0] * g.raise_t(t));
    const double as = fabs(t[1] * up[0] + t[2] * up[1] + t[3] * up[2]);
    if (!(at < 0.1 * as)) return false;
  }
  return true;
}

// The back-up equations of Sec. 4.11 for a zone that the energy methods left
// without a solution.  First the entropy equation (Eq. source6) in place of
// the gas energy equation, where the explicit S* (sqrt(-g) S u^t) is finite,
// by the energy methods' sequence: PMHD (emode 1; with emode 2 the update
// kernel ran it already and px / peT are its best iterate and error), then
// URAD and PRAD while the best entropy solution has e_T >= 1e-9, each from the
// primitives of that solution if its e_T < 1e-4, else from P_s.  Then, for a
// cold momentum-dominated zone (cold_allowed), the cold-MHD equations: PMHD
// on the three momentum equations with u_g held at the guess.  The PMHD
// attempts start from the energy PMHD's guess (P_s, or where tau < 2/3 the
// gas inversion of U*); a solution is accepted at e_T <= 1e-7.  Returns
// METH_ENTROPY (the entropy PMHD's solution), METH_ENTROPY_RAD (the entropy
// URAD's or PRAD's) or METH_COLD with Pn and *eT set, 0 if none gives a
// solution; adds the Newton steps to *steps.  emode 0: no entropy equation.
template <int MET>
__device__ int backup_equations(const DevParams& p, const Geo<MET, double>& g, const ImpSys<MET>& s,
                                const double Ust[NPR], const double Ps[NPR], double Sst, int emode,
                                double tau, double Pn[NPR], double* eT, int* steps,
                                const double* px = nullptr, double peT = HUGE_VAL) {
  const bool ent = emode != 0 && isfinite(Sst);
  const bool cold = cold_allowed<MET>(g, Ust, Ps);
  if (!ent && !cold) return 0;
  double x0[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
  if (tau < 2.0 / 3.0) {
    double go[5], T3[3] = {s.Ts[1], s.Ts[2], s.Ts[3]};
    if (gas_invert<MET>(p, g, s.Dlab, s.Ts[0], T3, s.B, Ps, 1e-9, go) == 0)
      for (int c = 0; c < 4; ++c) x0[c] = go[1 + c];
  }
  if (ent) {
    ImpSys<MET> se = s;
    se.entropy = true;
    se.Sstar = Sst / g.gdet;
    double bxe[4] = {0.0, 0.0, 0.0, 0.0}, beT = HUGE_VAL;
    int who = -1;  // 0 PMHD, 1 URAD, 2 PRAD
    if (emode == 1) {
      double xe[4] = {x0[0], x0[1], x0[2], x0[3]};
      entropy_ug_guess(p, Sst, s.Dlab * g.gdet, Ps[RHO], xe);
      *steps += newton_pmhd<MET>(p, se, xe, bxe, &beT);
    } else if (px && isfinite(peT)) {
      for (int c = 0; c < 4; ++c) bxe[c] = px[c];
      beT = peT;
    }
    if (isfinite(beT)) who = 0;
    double rx[2][4], rgas[2][5];
#pragma unroll 1
    for (int pr = 0; pr < 2 && !(beT < 1e-9); ++pr) {
      double Pq[NPR];
      for (int q = 0; q < NPR; ++q) Pq[q] = Ps[q];
      if (who >= 0 && beT < 1e-4) {
        if (who == 0) {
          ImpRes rr;
          ImpState stt;
          pmhd_res<MET>(p, se, bxe, rr, &stt, false);
          Pq[RHO] = stt.rho;
          for (int c = 0; c < 4; ++c) Pq[UU + c] = bxe[c];
          for (int c = 0; c < 4; ++c) Pq[ER + c] = stt.Pr[c];
        } else if (who == 1) {
          for (int c = 0; c < 5; ++c) Pq[c] = rgas[0][c];
          rad_invert<MET>(p, g, rx[0], 2, Pq + ER);
        } else {
          for (int c = 0; c < 5; ++c) Pq[c] = rgas[1][c];
          for (int c = 0; c < 4; ++c) Pq[ER + c] = rx[1][c];
        }
      }
      double gq[5] = {Pq[RHO], Pq[UU], Pq[U1], Pq[U2], Pq[U3]}, x4[4], reT;
      if (pr == 1) {
        for (int c = 0; c < 4; ++c) x4[c] = Pq[ER + c];
        *steps += newton_rad<MET, true>(p, se, x4, gq, rx[1], rgas[1], &reT);
      } else {
        double urc2[4], urv2[4], gr2;
        fourvel<MET, double>(g, Pq[UR1], Pq[UR2], Pq[UR3], urc2, urv2, &gr2);
        const double e43q = (4.0 / 3.0) * Pq[ER];
        x4[0] = e43q * urc2[0] * urv2[0] + Pq[ER] * (1.0 / 3.0);
        for (int c = 1; c < 4; ++c) x4[c] = e43q * urc2[0] * urv2[c];
        *steps += newton_rad<MET, false>(p, se, x4, gq, rx[0], rgas[0], &reT);
      }
      if (isfinite(reT) && (who < 0 || reT < beT)) {
        who = 1 + pr;
        beT = reT;
      }
    }
    if (beT <= 1e-7) {
      if (who == 0) {
        pmhd_final<MET>(p, se, bxe, Pn);
      } else {
        for (int q = 0; q < 5; ++q) Pn[q] = rgas[who - 1][q];
        if (who == 1) {
          double Pr[4];
          if (rad_invert<MET>(p, g, rx[0], 2, Pr)) rad_invert<MET>(p, g, rx[0], 0, Pr);
          for (int q = 0; q < 4; ++q) Pn[ER + q] = Pr[q];
        } else {
          for (int q = 0; q < 4; ++q) Pn[ER + q] = rx[1][q];
        }
        for (int c = 0; c < 3; ++c) Pn[B1 + c] = s.B[c];
      }
      *eT = beT;
      return who == 0 ? METH_ENTROPY : METH_ENTROPY_RAD;
    }
  }
  if (cold) {
    ImpSys<MET> sc = s;
    sc.entropy = false;
    sc.cold = true;
    double bxc[4] = {0.0, 0.0, 0.0, 0.0}, beT = HUGE_VAL;
    *steps += newton_pmhd<MET>(p, sc, x0, bxc, &beT);
    if (beT <= 1e-7) {
      pmhd_final<MET>(p, sc, bxc, Pn);
      *eT = beT;
      return METH_COLD;
    }
  }
  return 0;
}

// ------------------------------------------------------- update + implicit
// One thread per active zone: U(P_s), the geometric source
// SM_nu = 1/2 sqrt(-g) T^{mu kappa} d_nu g_{mu kappa}  (equal to
// sqrt(-g) T^kappa_lambda Gamma^lambda_{nu kappa} for a symmetric T, nonzero
// only for nu = x1, x2 on the stationary axisymmetric metric), the explicit
// update X = -sum_d dF_d/dx_d + SM, the RK3 combination
// U* = a_s U^n + b_s (U(P_s) + dt X) (Sec. 4.1), the PMHD Newton solve, floors.
// Zones whose PMHD error exceeds 1e-9 go to the retry queue, and so do zones
// whose radiation is extremely sub-dominant (URAD only, Sec. 4.10).
template <int MET, typename R, bool CONT, bool IMEX>
__device__ __forceinline__ void update_box(const DevParams& p, const BoxGeo& bx, int bi, const Bufs& b,
                                           int stage, int split, const ImexStage& im) {
  const double A = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
  const double Bc = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  {
    const double dt = b.dt[bi];
    double* P = b.P + 12 * bx.coff;
    const double* K = b.K + bx.coff;
    double* Un = b.Un + 12 * bx.aoff;
    const R* Fd[3] = {(const R*)b.F[0] + 12 * bx.coff, (const R*)b.F[1] + 12 * bx.coff,
                      (const R*)b.F[2] + 12 * bx.coff};
    const double idx[3] = {1.0 / bx.dx[0], 1.0 / bx.dx[1], 1.0 / bx.dx[2]};
    for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
      long long r = z;
      int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      int j = (int)(r % bx.n[1]);
      int k = (int)(r / bx.n[1]);
      long long t = cell_index(bx, i, j, k);
      double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
      const bool tab = MET == KS && b.geo && bx.goff >= 0;
      Geo<MET, double> g;
      MetricDeriv mdt;
      if (tab) {
        const GeoTab T = geotab(b.geo, bx);
        const long long gi = gidx_c(bx, i, j);
        g = geo_load<MET>(T.C, T.sC, gi);
        mdt = md_load(T.M, T.sC, gi);
      } else {
        g = make_geo<MET, double>(p, x1, x2);
      }
      double Ps[NPR];
#pragma unroll
      for (int q = 0; q < NPR; ++q) Ps[q] = P[q * bx.ntot + t];
      const double kz = kfield(p, K, t);
      double Us[NPR], X[NPR];
      cons_source<MET, double>(p, g, x1, x2, Ps, Us, X, tab ? &mdt : nullptr);
      // flux divergence (an IMEX stage without flux term reads no fluxes)
      const bool rhs = !IMEX || im.d != 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!p.act[d] || !rhs) continue;
        const long long s = bx.str[d];
#pragma unroll
        for (int q = 0; q < NPR; ++q) {
          R df = Fd[d][q * bx.ntot + t + s] - Fd[d][q * bx.ntot + t];
          X[q] -= double(df) * idx[d];
        }
      }
      double Ust[NPR];
#pragma unroll
      for (int q = 0; q < NPR; ++q) {
        double un;
        if (stage == 0) {
          Un[q * bx.nact + z] = Us[q];
          un = Us[q];
        } else {
          un = Un[q * bx.nact + z];
        }
        if constexpr (IMEX)
          Ust[q] = im.an * un + im.ap * Us[q] + im.d * dt * X[q];
        else
          Ust[q] = A * un + Bc * (Us[q] + dt * X[q]);
      }
      if (b.Bf[0]) {  // staggered field: B from the evolved faces (average of the two)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double* Bfd = b.Bf[d] + bx.coff;
          Ust[B1 + d] = p.act[d] ? 0.5 * (Bfd[t] + Bfd[t + bx.str[d]]) : Bfd[t];
        }
      }
      if (IMEX && stage > 0) {
        // earlier stages' implicit sources: +M on the gas rows, -M on the radiation rows
        const double* M = b.imexM + 16 * bx.aoff + z;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j >= stage) break;
          const double cj = im.c[j];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const double m = M[(4 * j + r) * bx.nact];
            Ust[UU + r] += dt * cj * m;
            Ust[ER + r] -= dt * cj * m;
          }
        }
      }
      if (b.ust_rec) {
#pragma unroll
        for (int q = 0; q < NPR; ++q) b.ust_rec[12 * bx.aoff + q * bx.nact + z] = Ust[q];
      }
      // RK3: the explicit entropy S* = a_s S^n + b_s (S(P_s) + dt X_S), the
      // conserved entropy sqrt(-g) S u^t = U_rho s_gas (Sec. 2, Eq. S), for the
      // entropy equation of the implicit solve (Sec. 4.7, 4.11); NaN: none
      double Sst = NAN;
      if (!IMEX && b.Sn) {
        const double Su = Us[RHO] * entropy_per_baryon<double>(p, Ps[RHO], Ps[UU]);
        double* Sn = b.Sn + bx.aoff;
        double sn;
        if (stage == 0) {
          Sn[z] = Su;
          sn = Su;
        } else {
          sn = Sn[z];
        }
        double divS = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (!p.act[d]) continue;
          const R* FSd = (const R*)b.FS[d] + bx.coff;
          divS += double(FSd[t + bx.str[d]] - FSd[t]) * idx[d];
        }
        Sst = A * sn + Bc * (Su - dt * divS);
        if (b.sst_rec) b.sst_rec[bx.aoff + z] = Sst;
      }
      // implicit solve
      const double h = IMEX ? im.g * dt : Bc * dt;
      // extremely sub-dominant radiation: no PMHD attempt; the zone goes to
      // the retry queue for URAD with a negative PMHD error as the mark
      const bool subdom = radiation_subdominant<MET>(g, Ust, Ps);
      ImpSys<MET> s;
      build_sys<MET>(p, g, Ust, h, kz, s);
      double x0[4] = {Ps[UU], Ps[U1], Ps[U2], Ps[U3]};
      {
        double kabs, ksca;
        opacity<double>(p, Ps[RHO], Ps[UU], kz, &kabs, &ksca);
        double dl = 0.0;
#pragma unroll
        for (int d = 1; d <= 3; ++d)
          if (p.act[d - 1]) dl = fmax(dl, sqrt(g.gdd(d)) * bx.dx[d - 1]);
        if ((kabs + ksca) * dl < 2.0 / 3.0) {
          double go[5];
          double T3[3] = {s.Ts[1], s.Ts[2], s.Ts[3]};
          if (gas_invert<MET>(p, g, s.Dlab, s.Ts[0], T3, s.B, Ps, 1e-9, go) == 0) {
            x0[0] = go[1];
            x0[1] = go[2];
            x0[2] = go[3];
            x0[3] = go[4];
          }
        }
      }
      bool accept = false;
      unsigned done_steps = 0;
      if (p.implicit_eq == 1) {
        // the entropy equation in every zone (Eq. source6), PMHD iterates;
        // e_T >= 1e-9 goes to the retry queue for the entropy URAD and PRAD
        // (the methods' sequence, Sec. 4.10-4.11)
        s.entropy = true;
        s.Sstar = Sst / g.gdet;
        double bxn[4] = {0.0, 0.0, 0.0, 0.0}, beT = HUGE_VAL;
        double xe[4] = {x0[0], x0[1], x0[2], x0[3]};
        entropy_ug_guess(p, Sst, s.Dlab * g.gdet, Ps[RHO], xe);
        const int steps = newton_pmhd<MET>(p, s, xe, bxn, &beT);
        accept = pmhd_finish<MET>(p, bx, bi, z, t, x1, g, s, Ust, h, bxn, beT, steps, P, b, Sst, 1e-9);
        done_steps = (unsigned)steps;
        warp_add(&b.stats[ST_ENTROPY], accept ? 1u : 0u);
      } else if constexpr (!CONT) {
        double bxn[4] = {0.0, 0.0, 0.0, 0.0}, beT = -1.0;
        ImpState bst;
        const int steps = subdom ? 0 : newton_pmhd<MET>(p, s, x0, bxn, &beT, &bst);
        accept = pmhd_finish<MET>(p, bx, bi, z, t, x1, g, s, Ust, h, bxn, beT, steps, P, b, Sst, 1e-9,
                                  subdom ? nullptr : &bst);
        done_steps = (unsigned)steps;
      } else {
        // the first `split` iterations here; a zone that needs more
        // continues in the compacted queue (k_newton_cont), so that the
        // heavy tail of iteration counts runs in full warps
        NewtonState ns;
        newton_pmhd_init(x0, ns);
        if (subdom) ns.best_eT = -1.0;
        if (subdom || newton_pmhd_run<MET>(p, s, ns, split)) {
          accept = pmhd_finish<MET>(p, bx, bi, z, t, x1, g, s, Ust, h, ns.best_x, ns.best_eT, ns.steps, P, b, Sst);
          done_steps = (unsigned)ns.steps;
        } else {
          const int slot = atomicAdd(&b.qcount[2], 1);
          b.czone[slot] = (int)z;
          b.cbox[slot] = bi;
          double* cd = b.cdata + (long long)slot * CSTRIDE;
#pragma unroll
          for (int q = 0; q < NPR; ++q) cd[q] = Ust[q];
          newton_state_store(ns, cd + NPR);
          cd[NPR + 22] = Sst;
        }
      }
      warp_add(&b.stats[ST_PMHD], accept ? 1u : 0u);
      warp_add(&b.stats[ST_ITERS], done_steps);
      warp_add(&b.stats[ST_SOLVES], 1u);
    }
  }
}

// Zones whose PMHD Newton iteration did not end within the update kernel's
// `split` iterations: a persistent grid over the compacted queue
// resumes each iteration from its saved state (same arithmetic as an
// uninterrupted iteration) and finishes the zone as the update kernel would.
template <int MET>
__global__ void __launch_bounds__(128) k_newton_cont(DevParams p, const BoxGeo* __restrict__ boxes, Bufs b,
                                                     double hfac) {
  const int nq = b.qcount[2];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nq; e += gridDim.x * blockDim.x) {
    const int bi = b.cbox[e];
    const BoxGeo& bx = boxes[bi];
    const long long z = b.czone[e];
    long long r = z;
    const int i = (int)(r % bx.n[0]);
    r /= bx.n[0];
    const int j = (int)(r % bx.n[1]);
    const int k = (int)(r / bx.n[1]);
    const long long t = cell_index(bx, i, j, k);
    const double x1 = xcen(bx, 0, i);
    const Geo<MET, double> g = geo_centre<MET, double>(p, bx, b.geo, i, j);
    const double* cd = b.cdata + (long long)e * CSTRIDE;
    double Ust[NPR];
    for (int q = 0; q < NPR; ++q) Ust[q] = cd[q];
    NewtonState ns;
    newton_state_load(cd + NPR, ns);
    const double h = hfac * b.dt[bi];  // the sub-step's implicit step fraction
    ImpSys<MET> s;
    build_sys<MET>(p, g, Ust, h, kfield(p, b.K + bx.coff, t), s);
    newton_pmhd_run<MET>(p, s, ns, 1 << 30);
    const bool accept = pmhd_finish<MET>(p, bx, bi, z, t, x1, g, s, Ust, h, ns.best_x, ns.best_eT, ns.steps,
                                         b.P + 12 * bx.coff, b, cd[NPR + 22]);
    if (accept) atomicAdd(&b.stats[ST_PMHD], 1ULL);
    atomicAdd(&b.stats[ST_ITERS], (unsigned long long)ns.steps);
  }
}

// IMEX: the sub-step of an IMEX scheme with coefficients im (otherwise RK3).
// ONE: a single grid whose geometry travels in the kernel's parameter space
// (no registers held for it across the Newton solve); otherwise the boxes of
// a batch, read from the device table.  CONT: PMHD iterations beyond `split`
// continue in k_newton_cont (the queue costs registers; it pays where the
// iteration counts are heavy-tailed, which the autotuner measures).
template <int MET, typename R, bool ONE, bool CONT, bool IMEX>
__global__ void __launch_bounds__(128) k_update(DevParams p, BoxGeo one, const BoxGeo* __restrict__ boxes,
                                                int nbox, Bufs b, int stage, int split, ImexStage im) {
  if constexpr (ONE) {
    update_box<MET, R, CONT, IMEX>(p, one, 0, b, stage, split, im);
  } else {
    for (int bi = 0; bi < nbox; ++bi) update_box<MET, R, CONT, IMEX>(p, boxes[bi], bi, b, stage, split, im);
  }
}

// IMEX: the implicit source of stage j on the gas rows,
// M^j = (U(P) - U*) / (g dt), with P the stage's implicit solution before the
// floors (the change the implicit stage made, Sec. 4.8); the radiation rows
// take -M^j, so gas plus radiation stays conserved.
template <int MET>
__global__ void k_imex_store(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, Bufs b, int j, double gj) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double h = gj * b.dt[bi];
    const double* Ps = b.psol_rec + 12 * bx.aoff;
    const double* Us = b.ust_rec + 12 * bx.aoff;
    double* M = b.imexM + 16 * bx.aoff;
    for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
      long long r = z;
      const int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      const int jj = (int)(r % bx.n[1]);
      const double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, jj);
      const Geo<MET, double> g = geo_centre<MET, double>(p, bx, b.geo, i, jj);
      double Pz[NPR], Uz[NPR], Xz[NPR];
#pragma unroll
      for (int q = 0; q < NPR; ++q) Pz[q] = Ps[q * bx.nact + z];
      cons_source<MET, double>(p, g, x1, x2, Pz, Uz, Xz, nullptr);
#pragma unroll
      for (int q = 0; q < 4; ++q) M[(4 * j + q) * bx.nact + z] = (Uz[UU + q] - Us[(UU + q) * bx.nact + z]) / h;
    }
  }
}

// ----------------------------------------------------------- retry (URAD)
// Persistent grid over the retry queue (its length is read on the device, so
// the launch needs no host round trip and can live in a CUDA graph): URAD,
// then PRAD (retry_sequence); e_T > 1e-7 sends the zone to the
// neighbour-average back-up.
template <int MET>
__global__ void __launch_bounds__(128) k_retry(DevParams p, const BoxGeo* __restrict__ boxes, Bufs b) {
  const int nq = b.qcount[0];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nq; e += gridDim.x * blockDim.x) {
    const long long z = b.qzone[e];
    const int bi = b.qbox[e];
    const BoxGeo& bx = boxes[bi];
    double* P = b.P + 12 * bx.coff;
    const double* K = b.K + bx.coff;
    const double* qd = b.qdata + (long long)e * QSTRIDE;
    long long r = z;
    int i = (int)(r % bx.n[0]);
    r /= bx.n[0];
    int j = (int)(r % bx.n[1]);
    int k = (int)(r / bx.n[1]);
    long long t = cell_index(bx, i, j, k);
    double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
    Geo<MET, double> g = make_geo<MET, double>(p, x1, x2);
    double Ust[NPR], Ps[NPR], px[4];
    for (int q = 0; q < NPR; ++q) {
      Ust[q] = qd[q];
      Ps[q] = P[q * bx.ntot + t];
    }
    for (int q = 0; q < 4; ++q) px[q] = qd[12 + q];
    // qd[16] < 0: radiation extremely sub-dominant, URAD only (no PMHD iterate)
    const bool subdom = qd[16] < 0.0;
    const double peT = subdom ? HUGE_VAL : qd[16];
    const double h = qd[17];
    ImpSys<MET> s;
    build_sys<MET>(p, g, Ust, h, kfield(p, K, t), s);
    const long long zg = bx.aoff + z;
    double Pn[NPR], eT;
    int steps;
    const double tau = zone_tau<MET>(p, g, bx.dx, Ps, kfield(p, K, t));
    int method;
    const double Sst = qd[18];
    if (p.implicit_eq == 1) {  // the entropy PMHD of the update kernel left e_T >= 1e-9
      for (int q = 0; q < NPR; ++q) Pn[q] = Ps[q];
      for (int c = 0; c < 3; ++c) Pn[B1 + c] = s.B[c];
      eT = HUGE_VAL;
      steps = 0;
      method = ST_BACKUP;
    } else {
      method = retry_sequence<MET>(p, g, s, Ps, px, peT, tau, Pn, &eT, &steps, subdom, Sst);
    }
    // no energy-based solution: the entropy, then the cold-MHD equations
    int by = 0;
    if (method == ST_BACKUP) {
      by = p.implicit_eq == 1 ? backup_equations<MET>(p, g, s, Ust, Ps, Sst, 2, tau, Pn, &eT, &steps, px, peT)
                              : backup_equations<MET>(p, g, s, Ust, Ps, Sst, 1, tau, Pn, &eT, &steps);
      // a retry method's solution, except that in the entropy-everywhere
      // mode the entropy PMHD is the first method
      if (by) method = (p.implicit_eq == 1 && by == METH_ENTROPY) ? ST_PMHD : ST_URAD;
    }
    b.iters[zg] += steps;
    if (b.psol_rec)
      for (int q = 0; q < NPR; ++q) b.psol_rec[12 * bx.aoff + q * bx.nact + z] = Pn[q];
    unsigned fcode = 0;
    apply_floors<MET>(p, g, log_r<MET>(p, x1), Pn, p.sig ? &fcode : nullptr);
    if (p.sig) sig_put(p, bx.coff + t, 60, fcode << 4 | (unsigned)method);
    for (int q = 0; q < NPR; ++q) P[q * bx.ntot + t] = Pn[q];
    unsigned char m = (unsigned char)method;
    if (m > b.status[zg]) b.status[zg] = m;
    // the adjoint differentiates every entropy solution through the entropy
    // PMHD's system (the URAD and PRAD solve the same equations)
    if (b.meth_rec) b.meth_rec[zg] = by ? (unsigned char)(by == METH_ENTROPY_RAD ? METH_ENTROPY : by) : m;
    if (by == METH_ENTROPY || by == METH_ENTROPY_RAD) atomicAdd(&b.stats[ST_ENTROPY], 1ULL);
    if (by == METH_COLD) atomicAdd(&b.stats[ST_COLD], 1ULL);
    if (method == ST_BACKUP || by == METH_COLD) {
      // the back-up average: all primitives but B, or u_g alone for a
      // cold-MHD solution (Sec. 4.11); either counts as not good for its
      // neighbours' averages
      b.failed[zg] = method == ST_BACKUP ? 1 : 2;
      int slot = atomicAdd(&b.qcount[1], 1);
      b.fzone[slot] = (int)z;
      b.fbox[slot] = bi;
    }
    if (method == ST_BACKUP) {
      atomicAdd(&b.stats[ST_BACKUP], 1ULL);
    } else if (method == ST_URAD) {
      atomicAdd(&b.stats[ST_URAD], 1ULL);
    } else {
      atomicAdd(&b.stats[ST_PMHD], 1ULL);
    }
    atomicAdd(&b.stats[ST_ITERS], (unsigned long long)steps);
  }
}

// ------------------------------------------------------------- back-up
// Average of the good active face neighbours (all active neighbours if none
// is good); B keeps its constrained-transport value, and a zone solved by the
// cold-MHD equations takes the average for u_g alone (Sec. 4.11).  All
// averages are formed before any is written back (k_backup_apply).
static __global__ void k_backup_avg(DevParams p, const BoxGeo* __restrict__ boxes, Bufs b) {
  const int nf = b.qcount[1];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf; e += gridDim.x * blockDim.x) {
    const BoxGeo& bx = boxes[b.fbox[e]];
    const double* P = b.P + 12 * bx.coff;
    long long z = b.fzone[e];
    long long r = z;
    int ii[3];
    ii[0] = (int)(r % bx.n[0]);
    r /= bx.n[0];
    ii[1] = (int)(r % bx.n[1]);
    ii[2] = (int)(r / bx.n[1]);
    double sg[NPR], sa[NPR];
    for (int q = 0; q < NPR; ++q) sg[q] = sa[q] = 0.0;
    int ng = 0, na = 0;
    for (int d = 0; d < 3; ++d) {
      if (bx.n[d] == 1) continue;
      for (int side = -1; side <= 1; side += 2) {
        int nb[3] = {ii[0], ii[1], ii[2]};
        nb[d] += side;
        if (nb[d] < 0 || nb[d] >= bx.n[d]) continue;
        long long zn = ((long long)nb[2] * bx.n[1] + nb[1]) * bx.n[0] + nb[0];
        long long tn = cell_index(bx, nb[0], nb[1], nb[2]);
        bool good = !b.failed[bx.aoff + zn];
        for (int q = 0; q < NPR; ++q) {
          double v = P[q * bx.ntot + tn];
          sa[q] += v;
          if (good) sg[q] += v;
        }
        ++na;
        if (good) ++ng;
      }
    }
    long long t = cell_index(bx, ii[0], ii[1], ii[2]);
    if (p.sig) sig_put(p, bx.coff + t, 61, (unsigned)ng << 4 | (unsigned)na);
    const bool cold = b.failed[bx.aoff + z] == 2;
    for (int q = 0; q < NPR; ++q) {
      double v = P[q * bx.ntot + t];
      if (na > 0 && !(q >= B1 && q <= B3) && (!cold || q == UU)) v = ng > 0 ? sg[q] / ng : sa[q] / na;
      b.ftmp[(long long)e * NPR + q] = v;
    }
  }
}

template <int MET>
__global__ void k_backup_apply(DevParams p, const BoxGeo* __restrict__ boxes, Bufs b) {
  const int nf = b.qcount[1];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf; e += gridDim.x * blockDim.x) {
    const BoxGeo& bx = boxes[b.fbox[e]];
    double* P = b.P + 12 * bx.coff;
    long long z = b.fzone[e];
    long long r = z;
    int i = (int)(r % bx.n[0]);
    r /= bx.n[0];
    int j = (int)(r % bx.n[1]);
    int k = (int)(r / bx.n[1]);
    long long t = cell_index(bx, i, j, k);
    double x1 = xcen(bx, 0, i), x2 = xcen(bx, 1, j);
    Geo<MET, double> g = make_geo<MET, double>(p, x1, x2);
    double Pn[NPR];
    for (int q = 0; q < NPR; ++q) Pn[q] = b.ftmp[(long long)e * NPR + q];
    unsigned fcode = 0;
    apply_floors<MET>(p, g, log_r<MET>(p, x1), Pn, p.sig ? &fcode : nullptr);
    if (p.sig) sig_put(p, bx.coff + t, 62, fcode);
    for (int q = 0; q < NPR; ++q) P[q * bx.ntot + t] = Pn[q];
  }
}

// --------------------------------------------------------------- CFL dt
// dt = C min_zones 1 / sum_d (v_d/dx_d), v_d = larger face speed of the zone
// along d, per grid.  Block minimum by warp shuffles, then one atomicMin on
// the bit pattern (positive doubles order like unsigned integers).
template <typename R>
__global__ void k_cfl(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, Bufs b) {
  __shared__ double sm[32];
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    double best = HUGE_VAL;
    for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
      long long r = z;
      int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      int j = (int)(r % bx.n[1]);
      int k = (int)(r / bx.n[1]);
      long long t = cell_index(bx, i, j, k);
      double sum = 0.0;
      for (int d = 0; d < 3; ++d) {
        if (bx.n[d] == 1) continue;
        const R* sp = (const R*)b.spd[d] + bx.coff;
        double v = fmax((double)sp[t], (double)sp[t + bx.str[d]]);
        sum += v / bx.dx[d];
      }
      if (sum > 0.0) best = fmin(best, 1.0 / sum);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = best;
    __syncthreads();
    if (w == 0) {
      best = lane < (int)(blockDim.x >> 5) ? sm[lane] : HUGE_VAL;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
      if (lane == 0 && best < HUGE_VAL)
        atomicMin(&b.dtmin[bi], (unsigned long long)__double_as_longlong(best));
    }
  }
}

static __global__ void k_cfl_init(Bufs b, int nbox) {
  for (int i = threadIdx.x; i < nbox; i += blockDim.x) b.dtmin[i] = 0x7FF0000000000000ULL;  // +inf
}

static __global__ void k_cfl_finish(DevParams p, Bufs b, int nbox) {
  for (int i = threadIdx.x; i < nbox; i += blockDim.x)
    b.dt[i] = p.courant * __longlong_as_double((long long)b.dtmin[i]);
}

}  // namespace hr
