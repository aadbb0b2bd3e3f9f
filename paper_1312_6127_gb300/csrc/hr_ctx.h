// Host-side context of the harmrad library (internal).
#pragma once
#include <cuda_runtime.h>

#include "../../include/harmrad.h"
#include "hr_common.cuh"

namespace hr {
struct Bufs;
struct AdjBufs;
}

struct harmrad_ctx {
  harmrad_params prm;        // parameters of the first grid
  hr::DevParams dp;          // physics shared by every grid
  int nbox;                  // grids in this context (1, or the boxes of a batch)
  hr::BoxGeo* boxes;         // host copy of the grid table
  hr::BoxGeo* dboxes;        // device copy
  long long ncell, nact;     // totals over the grids
  long long maxcell, maxact; // largest grid
  cudaStream_t stream;
  bool own_stream;
  int device;
  int sms;
  size_t real_size;  // 8 (FP64) or 4 (split)
  // device memory
  double* P;
  double* K;
  double* geotab;  // metric tables of Kerr-Schild grids (null for Minkowski)
  double* Un;
  double* Sn;   // [nact] conserved entropy sqrt(-g) S u^t at the start of the step (RK3)
  void* FS[3];  // [ntot] entropy face fluxes of each active direction (RK3; null otherwise)
  void* F[3];
  void* spd[3];
  void* aux;
  void* flat[3];
  void* emf;
  // staggered field (emf mode 1; null otherwise): sqrt(-g) B^d on the d-faces
  // and its value at the start of the step [ntot] each, gas signal speeds of
  // the faces [2][ntot] per direction, cell 3-velocities [3][ntot] and the
  // three edge EMFs [ntot] each (real type of the precision mode)
  double* Bf[3];
  double* Bfn[3];
  void* gsp[3];
  void* vel;
  void* emf3[3];
  void* edges;  // [2][12][ntot] reconstructed edge values of one direction
  void* slope;  // [12][ntot] MC slopes of one direction
  double* dt;
  unsigned char* status;
  int* iters;
  unsigned char* failed;
  int* qcount;
  int* czone;
  int* cbox;
  double* cdata;
  int* qzone;
  int* qbox;
  double* qdata;
  int* fzone;
  int* fbox;
  double* ftmp;
  unsigned long long* stats;
  unsigned long long* dtmin;
  double* stage_buf;      // [12][nact] active-layout staging for set/get
  int* flag;              // validation flag
  double* host_dt;        // pinned host scalar for dt read-back
  bool has_prims;
  // adjoint (harmrad_adjoint_enable): workspace, the saved input of the last
  // step, and the record pointers the forward kernels fill while the adjoint
  // recomputes that step
  hr::AdjBufs* adj;
  double* adj_Pn;
  bool adj_ready;  // a step has run since the adjoint was enabled
  double* rec_ust;
  unsigned char* rec_meth;
  double* rec_psol;
  double* rec_sst;
  double* imex_ust;   // IMEX: [12][nact] U* of the current stage
  double* imex_psol;  // IMEX: [12][nact] implicit solution of the current stage (before floors)
  double* imex_M;     // IMEX: [4 stages][4 gas rows][nact] implicit sources M^j
  // launch shapes of the heavy kernels (threads per block, resident-block cap
  // per SM of the grid-stride grid); chosen by harmrad_autotune
  harmrad_tuning tune;
  // CUDA graphs of a full step: [0] dt given, [1] CFL dt
  cudaGraphExec_t graph[2];
  bool use_graph;
  int launches_per_step;
  double last_dt;
  unsigned long long* sig;   // branch signature per cell (null unless enabled)
  // per-kernel profiling (harmrad_profile_step): an event after every launch
  bool profiling;
  int nev;
  cudaEvent_t ev[512];
  int ev_tag[512];
};

namespace hr {
// Record an event tagged with the kernel class after a launch (profiling only).
inline void mark(harmrad_ctx* c, int tag) {
  if (!c->profiling || c->nev >= 512) return;
  if (!c->ev[c->nev]) cudaEventCreate(&c->ev[c->nev]);
  c->ev_tag[c->nev] = tag;
  cudaEventRecord(c->ev[c->nev], c->stream);
  c->nev++;
}
}  // namespace hr

namespace hr {

// Launch sequences, instantiated per metric in hr_run_mink.cu / hr_run_ks.cu.
// Each returns the number of kernels it enqueued, or a negative error code.
template <int MET>
struct Run {
  static int faces(harmrad_ctx* c, bool fresh);     // ghosts, prep, flattener, fluxes, flux-CT
  static int cfl(harmrad_ctx* c);                   // faces(fresh) + reduction into *dt
  static int solve(harmrad_ctx* c, int stage, const ImexStage& im);  // update + implicit, retry, back-up
  // reverse sweep of the last step: gPout (device, active layout) -> gPin, gk
  static int adjoint(harmrad_ctx* c, const double* gPout, double* gPin, double* gk);
  static int zone_physics(const DevParams& dp, const BoxGeo& bg, int n, const double* x,
                          const double* P, double* U, double* SM, double* F, double* speeds,
                          cudaStream_t st, int sms);
  // staggered field: the faces from the cell-centred B (from_centres: after
  // a set of the primitives), then the ghost faces and the cell-centred B of
  // the active zones from the evolved faces
  static int init_faces(harmrad_ctx* c, bool from_centres);
  static int zone_method(const DevParams& dp, const BoxGeo& bg, int n, const double* x, const double* Us,
                         const double* Ss, const double* Ps, const double* h, int method, double* Pout,
                         double* eT, int* iters, cudaStream_t st, int sms);
  static int zone_implicit(const DevParams& dp, const BoxGeo& bg, int n, const double* x,
                           const double* Us, const double* Ss, const double* Ps, const double* h,
                           double* Pout, double* eT, int* iters, unsigned char* method, cudaStream_t st,
                           int sms);
};

}  // namespace hr
