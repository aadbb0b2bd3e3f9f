// Staggered magnetic field with the 4-state upwind EMF (Sec. 4, the list of
// quantities: B on cell faces, EMFs on the cell edges; Sec. 4.2 steps
// viii-x, after Del Zanna et al. 2007).  Used when the context's emf mode is
// HARMRAD_EMF_UCT; flux-CT (hr_kernels.cuh) otherwise.
//
// Bf[d] holds sqrt(-g) B^d on the lower d-face of every cell (ghosts
// included, the cell-indexed layout of the primitives); a direction with one
// zone has one face per cell, the cell itself.  The evolved faces are, along
// d, faces 0..n_d (0..n_d-1 on a periodic direction, where face n_d is the
// image of face 0) and, across, the active zones.  A zone's cell-centred
// sqrt(-g) B^d is the average of its two d-faces.
#pragma once
#include "hr_kernels.cuh"

namespace hr {

// sqrt(-g) at internal coordinates (x1, x2): the closed form of make_geo.
template <int MET>
__device__ __forceinline__ double gdet_at(const DevParams& p, double x1, double x2) {
  if constexpr (MET == MINK) {
    (void)p;
    (void)x1;
    (void)x2;
    return 1.0;
  } else {
    const double pi = 3.14159265358979323846;
    const double ex = exp(x1);
    const double r = p.R0 + ex;
    double s2x, c2x;
    sincospi(2.0 * x2, &s2x, &c2x);
    const double th = pi * x2 + 0.5 * (1.0 - p.h) * s2x;
    double sth, cth;
    sincos(th, &sth, &cth);
    const double S = r * r + p.a * p.a * cth * cth;
    return S * fabs(sth) * ex * (pi * (1.0 + (1.0 - p.h) * c2x)) * (2.0 * pi);
  }
}

// sqrt(-g) at a cell position (q0, q1) of the grid (ghosts included) whose
// x1 (f0) and/or x2 (f1) coordinate sits on the cell's lower face: from the
// Kerr-Schild metric tables (centres, x1 faces, x2 faces) where the context
// has them, else from the closed form.
template <int MET>
__device__ __forceinline__ double gdet_pos(const DevParams& p, const double* geo, const BoxGeo& bx, bool f0, bool f1,
                                           int q0, int q1) {
  f0 = f0 && bx.n[0] > 1;
  f1 = f1 && bx.n[1] > 1;
  if constexpr (MET == KS) {
    if (geo && bx.goff >= 0 && !(f0 && f1)) {
      const GeoTab T = geotab(geo, bx);
      if (f0) return __ldg(T.F0 + 13 * T.sF0 + gidx_f0(bx, q0, q1));
      if (f1) return __ldg(T.F1 + 13 * T.sF1 + gidx_f1(bx, q0, q1));
      return __ldg(T.C + 13 * T.sC + gidx_c(bx, q0, q1));
    }
  }
  const double x1 = f0 ? bx.x0[0] + q0 * bx.dx[0] : xcen(bx, 0, q0);
  const double x2 = f1 ? bx.x0[1] + q1 * bx.dx[1] : xcen(bx, 1, q1);
  return gdet_at<MET>(p, x1, x2);
}

__device__ __forceinline__ bool periodic_dir(const BoxGeo& bx, int d) {
  return bx.bc[2 * d] == 0 && bx.bc[2 * d + 1] == 0;
}
// internal coordinate of a cell's lower d-face (its centre when n_d = 1)
__device__ __forceinline__ double xface(const BoxGeo& bx, int d, int i) {
  return bx.n[d] > 1 ? bx.x0[d] + i * bx.dx[d] : xcen(bx, d, i);
}
// upper end of the evolved face range along e for faces of direction d
__device__ __forceinline__ int face_hi(const BoxGeo& bx, int d, int e) {
  return (e == d && bx.n[d] > 1 && !periodic_dir(bx, d)) ? bx.n[d] + 1 : bx.n[e];
}

struct FaceSet {
  double* f[3];
};

// Faces outside the evolved ranges: the periodic image where one exists,
// else the average of sqrt(-g) B^d of the two cells beside the face (the
// ghost cells hold the boundary conditions' B), or the one cell inside the
// array on the outermost layer.  Run after the ghost fill of P.
template <int MET>
__global__ void k_face_ghosts(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, const double* __restrict__ P0,
                              FaceSet F, int d, const double* __restrict__ geo) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    double* Bf = F.f[d] + bx.coff;
    const long long sd = bx.str[d];
    for (long long t = HR_TID; t < bx.ntot; t += HR_STRIDE) {
      long long r = t;
      int ii[3];
      ii[0] = (int)(r % bx.N[0]) - bx.ng[0];
      r /= bx.N[0];
      ii[1] = (int)(r % bx.N[1]) - bx.ng[1];
      ii[2] = (int)(r / bx.N[1]) - bx.ng[2];
      bool inside = true;
      for (int e = 0; e < 3; ++e) inside = inside && ii[e] >= 0 && ii[e] < face_hi(bx, d, e);
      if (inside) continue;
      int w[3] = {ii[0], ii[1], ii[2]};
      bool image = true;
      for (int e = 0; e < 3; ++e) {
        if (w[e] >= 0 && w[e] < face_hi(bx, d, e)) continue;
        if (periodic_dir(bx, e) && bx.n[e] > 1) w[e] = ((w[e] % bx.n[e]) + bx.n[e]) % bx.n[e];
        else image = false;
      }
      if (image) {
        Bf[t] = Bf[cell_index(bx, w[0], w[1], w[2])];
        continue;
      }
      const double bt = gdet_pos<MET>(p, geo, bx, false, false, ii[0], ii[1]) * P[(B1 + d) * bx.ntot + t];
      if (bx.n[d] == 1 || ii[d] == -bx.ng[d]) {
        Bf[t] = bt;
      } else {
        int m[3] = {ii[0], ii[1], ii[2]};
        m[d] -= 1;
        Bf[t] = 0.5 * (gdet_pos<MET>(p, geo, bx, false, false, m[0], m[1]) * P[(B1 + d) * bx.ntot + t - sd] + bt);
      }
    }
  }
}

// Every face from the cell-centred B (initialisation from primitives): the
// average of sqrt(-g) B^d of the two cells beside it.  Run after the ghost
// fill of P; k_face_ghosts and k_centre_B follow.
template <int MET>
__global__ void k_faces_from_centres(DevParams p, const BoxGeo* __restrict__ boxes, int nbox,
                                     const double* __restrict__ P0, FaceSet F, const double* __restrict__ geo) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    for (long long t = HR_TID; t < bx.ntot; t += HR_STRIDE) {
      long long r = t;
      int ii[3];
      ii[0] = (int)(r % bx.N[0]) - bx.ng[0];
      r /= bx.N[0];
      ii[1] = (int)(r % bx.N[1]) - bx.ng[1];
      ii[2] = (int)(r / bx.N[1]) - bx.ng[2];
      const double gt = gdet_pos<MET>(p, geo, bx, false, false, ii[0], ii[1]);
      for (int d = 0; d < 3; ++d) {
        const double bt = gt * P[(B1 + d) * bx.ntot + t];
        double v = bt;
        if (bx.n[d] > 1 && ii[d] > -bx.ng[d]) {
          int m[3] = {ii[0], ii[1], ii[2]};
          m[d] -= 1;
          v = 0.5 * (gdet_pos<MET>(p, geo, bx, false, false, m[0], m[1]) * P[(B1 + d) * bx.ntot + t - bx.str[d]] + bt);
        }
        F.f[d][bx.coff + t] = v;
      }
    }
  }
}

// Cell-centred B of the active zones from their faces.
template <int MET>
__global__ void k_centre_B(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, double* __restrict__ P0,
                           FaceSet F, const double* __restrict__ geo) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    double* P = P0 + 12 * bx.coff;
    for (long long z = HR_TID; z < bx.nact; z += HR_STRIDE) {
      long long r = z;
      const int i = (int)(r % bx.n[0]);
      r /= bx.n[0];
      const int j = (int)(r % bx.n[1]);
      const int k = (int)(r / bx.n[1]);
      const long long t = cell_index(bx, i, j, k);
      const double ig = 1.0 / gdet_pos<MET>(p, geo, bx, false, false, i, j);
      for (int d = 0; d < 3; ++d) {
        const double* Bf = F.f[d] + bx.coff;
        const double c = bx.n[d] > 1 ? 0.5 * (Bf[t] + Bf[t + bx.str[d]]) : Bf[t];
        P[(B1 + d) * bx.ntot + t] = c * ig;
      }
    }
  }
}

// Lab-frame 3-velocity v^i = u^i / u^t of every cell, ghosts included.
template <int MET, typename R>
__global__ void k_vel(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, const double* __restrict__ P0,
                      R* __restrict__ V0, const double* __restrict__ geo) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double* P = P0 + 12 * bx.coff;
    R* V = V0 + 3 * bx.coff;
    for (long long t = HR_TID; t < bx.ntot; t += HR_STRIDE) {
      long long r = t;
      const int i = (int)(r % bx.N[0]) - bx.ng[0];
      r /= bx.N[0];
      const int j = (int)(r % bx.N[1]) - bx.ng[1];
      Geo<MET, double> g;
      bool tab = false;
      if constexpr (MET == KS) {
        if (geo && bx.goff >= 0) {
          const GeoTab T = geotab(geo, bx);
          g = geo_load<MET>(T.C, T.sC, gidx_c(bx, i, j));
          tab = true;
        }
      }
      if (!tab) g = make_geo<MET, double>(p, xcen(bx, 0, i), xcen(bx, 1, j));
      double ucon[4], ucov[4], gm;
      fourvel<MET, double>(g, P[U1 * bx.ntot + t], P[U2 * bx.ntot + t], P[U3 * bx.ntot + t], ucon, ucov, &gm);
      const double iut = 1.0 / ucon[0];
      for (int c = 0; c < 3; ++c) V[c * bx.ntot + t] = R(ucon[c + 1] * iut);
    }
  }
}

// The 4-state upwind EMF of the pair a < b (one of them with more than one
// zone) on the edges (lower a-face, lower b-face) of the cells:
// emf_ab = sqrt(-g) (B^b v^a - B^a v^b), the flux of sqrt(-g) B^b along a and
// minus that of sqrt(-g) B^a along b.  B^b comes from the b-faces on either
// side of the edge along a, interpolated to it along a (MC-limited linear),
// B^a likewise along b; the velocities of the four cells around the edge are
// extrapolated to it with MC-limited slopes.  The signal speeds along a
// average the gas speeds (v_max, v_min) of the two a-faces beside the edge,
// and likewise along b.  The four states are weighted as in the 2D HLL (LAXF:
// equal weights v_tot), with each direction's 1D HLL/LAXF dissipation
// (Eqs. hll, lax).  Edges on the polar axis carry no EMF.
template <int MET, typename R>
__global__ void k_uct_emf(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, FaceSet F,
                          const R* __restrict__ V0, const R* __restrict__ gsa0, const R* __restrict__ gsb0,
                          R* __restrict__ emf0, int a, int b, const double* __restrict__ geo) {
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const bool aa = bx.n[a] > 1, ab = bx.n[b] > 1;
    if (!aa && !ab) continue;
    const R* V = V0 + 3 * bx.coff;
    const R* gsa = gsa0 + 2 * bx.coff;
    const R* gsb = gsb0 + 2 * bx.coff;
    const double* Fa = F.f[a] + bx.coff;
    const double* Fb = F.f[b] + bx.coff;
    R* emf = emf0 + bx.coff;
    int len[3];
    for (int e = 0; e < 3; ++e) len[e] = bx.n[e] + (((e == a && aa) || (e == b && ab)) ? 1 : 0);
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
      if (MET == KS && (a == 1 || b == 1) &&
          ((ii[1] == 0 && bx.bc[2] == 2) || (ii[1] == bx.n[1] && bx.bc[3] == 2))) {
        emf[t] = R(0);
        continue;
      }
      // B^d at the face of the cell offset by o along m: Bf / sqrt(-g) there
      auto Bat = [&](const double* Fd, int d, int m, int o) {
        int q[3] = {ii[0], ii[1], ii[2]};
        q[m] += o;
        return Fd[t + o * bx.str[m]] / gdet_pos<MET>(p, geo, bx, d == 0, d == 1, q[0], q[1]);
      };
      double Bb[2], Ba[2];
      {
        const double b0 = Bat(Fb, b, a, 0);
        if (aa) {
          const double bmm = Bat(Fb, b, a, -2), bm = Bat(Fb, b, a, -1), bp = Bat(Fb, b, a, 1);
          Bb[0] = bm + 0.5 * mc_slope<double>(bmm, bm, b0);
          Bb[1] = b0 - 0.5 * mc_slope<double>(bm, b0, bp);
        } else {
          Bb[0] = Bb[1] = b0;
        }
      }
      {
        const double b0 = Bat(Fa, a, b, 0);
        if (ab) {
          const double bmm = Bat(Fa, a, b, -2), bm = Bat(Fa, a, b, -1), bp = Bat(Fa, a, b, 1);
          Ba[0] = bm + 0.5 * mc_slope<double>(bmm, bm, b0);
          Ba[1] = b0 - 0.5 * mc_slope<double>(bm, b0, bp);
        } else {
          Ba[0] = Ba[1] = b0;
        }
      }
      const double ge = gdet_pos<MET>(p, geo, bx, a == 0 || b == 0, a == 1 || b == 1, ii[0], ii[1]);
      double es[2][2];
#pragma unroll
      for (int s1 = 0; s1 < 2; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const long long tc = t - (s1 == 0 && aa ? sa : 0) - (s2 == 0 && ab ? sb : 0);
          double v[2];
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            const R* Vm = V + (m == 0 ? a : b) * bx.ntot;
            double val = double(Vm[tc]);
            if (aa) val += (s1 == 0 ? 0.5 : -0.5) * double(mc_slope<R>(Vm[tc - sa], Vm[tc], Vm[tc + sa]));
            if (ab) val += (s2 == 0 ? 0.5 : -0.5) * double(mc_slope<R>(Vm[tc - sb], Vm[tc], Vm[tc + sb]));
            v[m] = val;
          }
          es[s1][s2] = ge * (Bb[s1] * v[0] - Ba[s2] * v[1]);
        }
      double wa[2] = {0.0, 0.0}, wb[2] = {0.0, 0.0};
      if (aa) {
        const long long f0 = ab ? t - sb : t;
        const double vmax = 0.5 * (double(gsa[f0]) + double(gsa[t]));
        const double vmin = 0.5 * (double(gsa[bx.ntot + f0]) + double(gsa[bx.ntot + t]));
        if (p.flux == 0) {
          wa[0] = wa[1] = fmax(vmax, vmin);
        } else {
          wa[0] = vmax;
          wa[1] = vmin;
        }
      }
      if (ab) {
        const long long f0 = aa ? t - sa : t;
        const double vmax = 0.5 * (double(gsb[f0]) + double(gsb[t]));
        const double vmin = 0.5 * (double(gsb[bx.ntot + f0]) + double(gsb[bx.ntot + t]));
        if (p.flux == 0) {
          wb[0] = wb[1] = fmax(vmax, vmin);
        } else {
          wb[0] = vmax;
          wb[1] = vmin;
        }
      }
      double Wa = wa[0] + wa[1], Wb = wb[0] + wb[1], da = 0.0, db = 0.0;
      if (Wa > 0.0) {
        da = wa[0] * wa[1] / Wa;
      } else {
        wa[0] = wa[1] = 1.0;
        Wa = 1.0;
      }
      if (Wb > 0.0) {
        db = wb[0] * wb[1] / Wb;
      } else {
        wb[0] = wb[1] = 1.0;
        Wb = 1.0;
      }
      double sum = 0.0;
#pragma unroll
      for (int s1 = 0; s1 < 2; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) sum += wa[s1] * wb[s2] * es[s1][s2];
      emf[t] = R(sum / (Wa * Wb) - da * ge * (Bb[1] - Bb[0]) + db * ge * (Ba[1] - Ba[0]));
    }
  }
}

struct EmfSet {
  const void* e[3];  // emf_12 (index 2), emf_02 (index 1), emf_01 (index 0): e[3 - a - b]
};

// The evolved faces' stage: d(sqrt(-g) B^d)/dt = - sum_{a != d} d_a emf_{a d}
// (emf_{a d} = -emf_{d a}), combined with the step's initial faces like the
// cell-centred conserved quantities (RK3 stage coefficients, or an IMEX
// stage's an, ap, d); rhs = false: no EMF term (an IMEX stage without
// explicit right-hand side).  Bfn takes the faces at stage 0.
template <typename R>
__global__ void k_face_update(DevParams p, const BoxGeo* __restrict__ boxes, int nbox, FaceSet F, FaceSet Fn,
                              EmfSet E, const double* __restrict__ dt0, int stage, ImexStage im, bool rhs, int d) {
  const double A = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
  const double Bc = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  for (int bi = 0; bi < nbox; ++bi) {
    const BoxGeo& bx = boxes[bi];
    const double dt = dt0[bi];
    double* Bf = F.f[d] + bx.coff;
    double* Bn = Fn.f[d] + bx.coff;
    int len[3];
    for (int e = 0; e < 3; ++e) len[e] = face_hi(bx, d, e);
    const long long total = (long long)len[0] * len[1] * len[2];
    for (long long id = HR_TID; id < total; id += HR_STRIDE) {
      long long r = id;
      int ii[3];
      ii[0] = (int)(r % len[0]);
      r /= len[0];
      ii[1] = (int)(r % len[1]);
      ii[2] = (int)(r / len[1]);
      const long long t = cell_index(bx, ii[0], ii[1], ii[2]);
      double x = 0.0;
      if (rhs) {
        for (int a = 0; a < 3; ++a) {
          if (a == d || bx.n[a] == 1) continue;
          const R* em = (const R*)E.e[3 - a - d] + bx.coff;
          const double sgn = a < d ? 1.0 : -1.0;
          x -= sgn * double(em[t + bx.str[a]] - em[t]) / bx.dx[a];
        }
      }
      const double bs = Bf[t];
      if (stage == 0) Bn[t] = bs;
      const double bn = stage == 0 ? bs : Bn[t];
      Bf[t] = im.on ? im.an * bn + im.ap * bs + im.d * dt * x : A * bn + Bc * (bs + dt * x);
    }
  }
}

// Copy between the evolved-face layout of a single grid (direction d:
// [n3'][n2'][n1'], n_d' = n_d + 1 when n_d > 1, else 1) and the cell-indexed
// face arrays.  to_cells = true writes the faces.
static __global__ void k_face_pack(const BoxGeo* __restrict__ boxes, double* __restrict__ flat, FaceSet F,
                                   bool to_cells) {
  const BoxGeo& bx = boxes[0];
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    int m[3];
    for (int e = 0; e < 3; ++e) m[e] = bx.n[e] + ((e == d && bx.n[d] > 1) ? 1 : 0);
    const long long total = (long long)m[0] * m[1] * m[2];
    for (long long l = HR_TID; l < total; l += HR_STRIDE) {
      long long r = l;
      const int i = (int)(r % m[0]);
      r /= m[0];
      const int j = (int)(r % m[1]);
      const int k = (int)(r / m[1]);
      const long long t = cell_index(bx, i, j, k);
      if (to_cells) F.f[d][t] = flat[off + l];
      else flat[off + l] = F.f[d][t];
    }
    off += total;
  }
}

}  // namespace hr
