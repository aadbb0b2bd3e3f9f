// harmrad_zone_implicit_static: the per-zone implicit solve with its retry
// queue in statically allocated device memory, for callers that cannot
// allocate device memory.
//
// The solve runs in two kernels, like the grid step: a PMHD pass over all
// zones, which writes the zones it accepts and appends the others to a
// retry queue; then a URAD pass that drains the queue.  Here the queue lives
// in a file-scope __device__ array of fixed size, so a call makes no
// cudaMalloc/cudaFree and no allocating library call.  The array exists once
// per device that loads the library and lives until the process exits.
#include <cuda_runtime.h>
#include <math.h>

#include <atomic>
#include <mutex>

#include "../../include/harmrad.h"
#include "hr_common.cuh"
#include "hr_implicit.cuh"
#include "hr_kernels.cuh"

namespace {

// Largest zone count one call accepts; the queue below is sized for it.
constexpr int kStaticMaxZones = 65536;

// Queue layout (bytes): [0, 256) header with the entry counter;
// then kStaticMaxZones int zone indices; then kStaticMaxZones records of
// 5 doubles (PMHD best iterate x[4] and its e_T).
constexpr size_t kHeader = 256;
constexpr size_t kIdxBytes = sizeof(int) * kStaticMaxZones;
constexpr size_t kRecBytes = sizeof(double) * 5 * kStaticMaxZones;
constexpr size_t kScratchBytes = kHeader + kIdxBytes + kRecBytes;  // about 2.9 MB

static __device__ __align__(256) unsigned char g_zi_scratch[kScratchBytes];

// Device address of g_zi_scratch, looked up once per device and context (host
// code may not use the symbol itself: on the host it names a stand-in, not
// device memory).  The address belongs to the module loaded in the device's
// current context; a device reset destroys that context and the next one
// loads the module again, possibly elsewhere.  So each entry remembers the
// unique id of the context it was looked up in, and a call made in another
// context looks the address up again.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  std::atomic<unsigned long long> ctx_id{0};  // 0: not looked up yet
  std::atomic<void*> addr{nullptr};
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Driver entry points for the current context's id, reached through the
// runtime (no link against the driver library).
using PfnCtxGetCurrent = int (*)(void**);
using PfnCtxGetId = int (*)(void*, unsigned long long*);

int current_context_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (PfnCtxGetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (PfnCtxGetId)f;
    cudaGetLastError();
  });
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0 || *id == 0)
    return HARMRAD_E_CUDA;
  return HARMRAD_OK;
}

struct QueueView {
  int* count;
  int* idx;
  double* rec;
};

__host__ __device__ inline QueueView queue_view(void* base) {
  unsigned char* b = (unsigned char*)base;
  QueueView q;
  q.count = (int*)b;
  q.idx = (int*)(b + kHeader);
  q.rec = (double*)(b + kHeader + kIdxBytes);
  return q;
}

__global__ void k_zi_clear(void* base) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *queue_view(base).count = 0;
}

// Geometry, explicit state and the PMHD guess of one zone.
template <int MET>
__device__ void zi_setup(const hr::DevParams& p, int z, const double* x, const double* Us,
                         const double* Ps, const double* hh, hr::Geo<MET, double>& g,
                         hr::ImpSys<MET>& s, double P0[hr::NPR]) {
  using namespace hr;
  double x1 = x[4 * z + 1], x2 = x[4 * z + 2];
  g = make_geo<MET, double>(p, x1, x2);
  double Ust[NPR];
  for (int q = 0; q < NPR; ++q) {
    Ust[q] = Us[NPR * z + q];
    P0[q] = Ps[NPR * z + q];
  }
  build_sys<MET>(p, g, Ust, hh[z], 1.0, s);
}

template <int MET>
__global__ void k_zi_pmhd(hr::DevParams p, hr::BoxGeo bg, int n, const double* __restrict__ x,
                          const double* __restrict__ Us, const double* __restrict__ Ps,
                          const double* __restrict__ hh, double* Pout, double* eTo, int* itso,
                          unsigned char* meth, void* base) {
  using namespace hr;
  QueueView qv = queue_view(base);
  for (int z = blockIdx.x * blockDim.x + threadIdx.x; z < n; z += gridDim.x * blockDim.x) {
    Geo<MET, double> g;
    ImpSys<MET> s;
    double P0[NPR];
    zi_setup<MET>(p, z, x, Us, Ps, hh, g, s, P0);
    double x0[4] = {P0[UU], P0[U1], P0[U2], P0[U3]};
    double kabs, ksca;
    opacity<double>(p, P0[RHO], P0[UU], 1.0, &kabs, &ksca);
    double dl = 0.0;
    for (int d = 1; d <= 3; ++d)
      if (p.act[d - 1]) dl = fmax(dl, sqrt(g.gdd(d)) * bg.dx[d - 1]);
    if ((kabs + ksca) * dl < 2.0 / 3.0) {
      double go[5], T3[3] = {s.Ts[1], s.Ts[2], s.Ts[3]};
      if (gas_invert<MET>(p, g, s.Dlab, s.Ts[0], T3, s.B, P0, 1e-9, go) == 0) {
        x0[0] = go[1];
        x0[1] = go[2];
        x0[2] = go[3];
        x0[3] = go[4];
      }
    }
    double bx[4] = {0.0, 0.0, 0.0, 0.0}, beT = HUGE_VAL;
    // extremely sub-dominant radiation (Sec. 4.10): no PMHD attempt
    int steps = radiation_subdominant<MET>(g, Us + NPR * (size_t)z, P0) ? 0 : newton_pmhd<MET>(p, s, x0, bx, &beT);
    if (itso) itso[z] = steps;
    if (beT < 1e-9) {
      double Pn[NPR];
      pmhd_final<MET>(p, s, bx, Pn);
      for (int q = 0; q < NPR; ++q) Pout[NPR * z + q] = Pn[q];
      if (eTo) eTo[z] = beT;
      if (meth) meth[z] = 0;
    } else {
      int slot = atomicAdd(qv.count, 1);
      qv.idx[slot] = z;
      double* r = qv.rec + 5 * (size_t)slot;
      for (int q = 0; q < 4; ++q) r[q] = isfinite(beT) ? bx[q] : 0.0;
      r[4] = beT;
    }
  }
}

template <int MET>
__global__ void k_zi_urad(hr::DevParams p, hr::BoxGeo bg, const double* __restrict__ x,
                          const double* __restrict__ Us, const double* __restrict__ Ps,
                          const double* __restrict__ hh, double* Pout, double* eTo, int* itso,
                          unsigned char* meth, void* base) {
  using namespace hr;
  QueueView qv = queue_view(base);
  const int nq = *qv.count;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nq; e += gridDim.x * blockDim.x) {
    const int z = qv.idx[e];
    const double* r = qv.rec + 5 * (size_t)e;
    Geo<MET, double> g;
    ImpSys<MET> s;
    double P0[NPR];
    zi_setup<MET>(p, z, x, Us, Ps, hh, g, s, P0);
    double bx[4] = {r[0], r[1], r[2], r[3]};
    const double beT = r[4];
    double Pn[NPR], eT;
    int steps;
    const double tau = zone_tau<MET>(p, g, bg.dx, P0, 1.0);
    const bool subdom = radiation_subdominant<MET>(g, Us + NPR * (size_t)z, P0);
    int method = retry_sequence<MET>(p, g, s, P0, bx, beT, tau, Pn, &eT, &steps, subdom);
    if (method == ST_BACKUP) {  // the cold-MHD equations (no explicit entropy here)
      const int by = backup_equations<MET>(p, g, s, Us + NPR * (size_t)z, P0, NAN, 0, tau, Pn, &eT, &steps);
      if (by) method = by;
    }
    for (int q = 0; q < NPR; ++q) Pout[NPR * z + q] = Pn[q];
    if (eTo) eTo[z] = eT;
    if (itso) itso[z] += steps;
    if (meth) meth[z] = (unsigned char)method;
  }
}

// Device address of the static queue on the current device (set-up on the
// first call in each context of the device).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return HARMRAD_E_ARG;
  // bind the device's primary context to this thread (it exists already: the
  // caller's buffers live in it), so that the driver reports it as current
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  ScratchAddr& e = g_scratch_addr[dev];
  if (e.ctx_id.load(std::memory_order_acquire) != id) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (e.ctx_id.load(std::memory_order_acquire) != id) {
      void* a = nullptr;
      if (cudaGetSymbolAddress(&a, g_zi_scratch) != cudaSuccess || !a) {
        cudaGetLastError();
        return HARMRAD_E_CUDA;
      }
      e.addr.store(a, std::memory_order_release);
      e.ctx_id.store(id, std::memory_order_release);
    }
  }
  *out = e.addr.load(std::memory_order_acquire);
  return HARMRAD_OK;
}

}  // namespace

extern int harmrad_fill_params_internal(const harmrad_params* p, hr::DevParams& d);
extern int harmrad_fill_geometry_internal(const harmrad_params* p, hr::BoxGeo& b);

extern "C" int harmrad_zone_implicit_static(const harmrad_params* prm, int n, const double* x,
                                            const double* Us, const double* Ps, const double* h,
                                            double* Pout, double* eT, int* iters,
                                            unsigned char* method, void* stream) {
  if (!prm || n < 0 || (n > 0 && (!x || !Us || !Ps || !h || !Pout))) return HARMRAD_E_ARG;
  if (n > kStaticMaxZones) return HARMRAD_E_ARG;
  hr::DevParams dp;
  hr::BoxGeo bg;
  int rc = harmrad_fill_params_internal(prm, dp);
  if (!rc) rc = harmrad_fill_geometry_internal(prm, bg);
  if (rc) return rc;
  if (dp.opacity == HARMRAD_OPAC_FIELD) return HARMRAD_E_ARG;
  if (n == 0) return HARMRAD_OK;
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_zi_clear<<<1, 32, 0, st>>>(base);
  int grid = hr::grid_for(n, sms, 128);
  if (dp.metric == 1) {
    k_zi_pmhd<hr::KS><<<grid, 128, 0, st>>>(dp, bg, n, x, Us, Ps, h, Pout, eT, iters, method, base);
    k_zi_urad<hr::KS><<<sms * 2, 128, 0, st>>>(dp, bg, x, Us, Ps, h, Pout, eT, iters, method, base);
  } else {
    k_zi_pmhd<hr::MINK><<<grid, 128, 0, st>>>(dp, bg, n, x, Us, Ps, h, Pout, eT, iters, method, base);
    k_zi_urad<hr::MINK><<<sms * 2, 128, 0, st>>>(dp, bg, x, Us, Ps, h, Pout, eT, iters, method, base);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  return HARMRAD_OK;
}
