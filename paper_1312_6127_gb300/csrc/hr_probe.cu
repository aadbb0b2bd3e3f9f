// harmrad_fp64_fma_rate: the FP64 fused multiply-add issue rate of the current
// device, measured with a kernel of independent FMA chains.  It is the
// denominator of the roofline fraction of the FP64-bound kernels (the update
// kernel spends its time on the FP64 pipe, not on memory).
//
// Each thread runs kChains independent recurrences a <- a b + c (one DFMA
// each, no dependency between chains), so the pipe, not the FMA latency,
// bounds the rate.  With b slightly below one and c small the values stay
// bounded; the sum of the chains is written so that nothing is eliminated.
#include <cuda_runtime.h>

#include "../../include/harmrad.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kBlock) k_dfma_chains(const double* __restrict__ bc, double* out, int iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double b = bc[0], c = bc[1];
  double a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = 1e-9 * t + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  out[t] = s;
}

}  // namespace

extern "C" int harmrad_fp64_fma_rate(int reps, double* tflops, void* stream) {
  if (!tflops || reps < 1 || reps > 100) return HARMRAD_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = sms * kBlocksPerSm;
  const long long threads = (long long)grid * kBlock;
  const int iters = 4096;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (2 + threads)) != cudaSuccess) {
    cudaGetLastError();
    return HARMRAD_E_OOM;
  }
  const double hbc[2] = {0.9999999, 1e-7};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HARMRAD_OK;
  float best = 0.0f;
  if (cudaMemcpyAsync(buf, hbc, sizeof(hbc), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = HARMRAD_E_CUDA;
  } else {
    k_dfma_chains<<<grid, kBlock, 0, st>>>(buf, buf + 2, iters);  // warm-up
    for (int r = 0; r < reps && rc == HARMRAD_OK; ++r) {
      float ms = 0.0f;
      if (cudaEventRecord(e0, st) != cudaSuccess) rc = HARMRAD_E_CUDA;
      k_dfma_chains<<<grid, kBlock, 0, st>>>(buf, buf + 2, iters);
      if (rc || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = HARMRAD_E_CUDA;
      else if (best == 0.0f || ms < best)
        best = ms;
    }
  }
  if (cudaGetLastError() != cudaSuccess) rc = HARMRAD_E_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc == HARMRAD_OK) {
    const double flops = 2.0 * kChains * (double)iters * (double)threads;
    *tflops = best > 0.0f ? flops / (best * 1e-3) / 1e12 : 0.0;
  }
  return rc;
}
