// Index helpers and constants shared by the kernels and the host code.
#pragma once
#include "hr_phys.cuh"

namespace hr {

enum { ST_PMHD = 0, ST_URAD = 1, ST_BACKUP = 2, ST_SOLVES = 3, ST_ITERS = 4 };
constexpr int QSTRIDE = 18;

__device__ __forceinline__ long long cell_index(const DevParams& p, int i, int j, int k) {
  return ((long long)(k + p.ng[2]) * p.N[1] + (j + p.ng[1])) * p.N[0] + (i + p.ng[0]);
}
__device__ __forceinline__ double xcen(const DevParams& p, int d, int i) {
  return p.x0[d] + (i + 0.5) * p.dx[d];
}

inline int grid_for(long long work, int sms, int block) {
  long long g = (work + block - 1) / block;
  long long cap = (long long)sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace hr
