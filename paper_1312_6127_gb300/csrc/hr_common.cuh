// Index helpers and constants shared by the kernels and the host code.
#pragma once
#include "hr_phys.cuh"

namespace hr {

enum { ST_PMHD = 0, ST_URAD = 1, ST_BACKUP = 2, ST_SOLVES = 3, ST_ITERS = 4, ST_ENTROPY = 5, ST_COLD = 6 };
// codes of a zone solved by the entropy equation (by the entropy PMHD, or by
// the entropy-based URAD or PRAD: METH_ENTROPY_RAD, which the adjoint record
// stores as METH_ENTROPY) or by the cold-MHD equations; their status byte is
// that of a retry method, ST_URAD, except for the entropy PMHD's solution in
// the entropy-everywhere mode, ST_PMHD
constexpr unsigned char METH_ENTROPY = 3;
constexpr unsigned char METH_COLD = 4;
constexpr unsigned char METH_ENTROPY_RAD = 5;
constexpr int QSTRIDE = 19;

// Coefficients of one sub-step of an IMEX scheme (Sec. 4.1, Eqs. IMEX2,
// IMEX2B, IMEX3) in its bracket form: U* = an U^n + ap U(P) + d dt F(P)
// + dt sum_j c_j M^j, then the implicit solve with step g dt (g = 0: the
// final combination, inverted only).  on = 0: the RK3 stage coefficients.
struct ImexStage {
  double an, ap, d, c[4], g;
  int on;
};

// Index of cell (i, j, k) (active indices, ghosts negative or >= n) within
// its grid's block of a cell-indexed array.
__host__ __device__ __forceinline__ long long cell_index(const BoxGeo& b, int i, int j, int k) {
  return ((long long)(k + b.ng[2]) * b.N[1] + (j + b.ng[1])) * b.N[0] + (i + b.ng[0]);
}
__host__ __device__ __forceinline__ double xcen(const BoxGeo& b, int d, int i) {
  return b.x0[d] + (i + 0.5) * b.dx[d];
}

inline int grid_for(long long work, int sms, int block, int per_sm = 16) {
  long long g = (work + block - 1) / block;
  long long cap = (long long)sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace hr
