// fslbm_rate.cu -- the FP64 arithmetic rate of the device, the ceiling of the
// FP64 form where its stream-collide is bound by arithmetic, not by memory.
#include <cuda_runtime.h>

#include "fslbm.h"

namespace {

// Eight independent chains of dependent fused multiply-adds per thread (no
// memory traffic inside the loop; the result is stored so that the chains
// are not removed).
__global__ void __launch_bounds__(256) k_dfma(int iters, double a, double b, double* out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;  // (never true for these inputs; keeps the work)
}

}  // namespace

extern "C" int fslbm_fp64_rate(double* tflops, void* stream) {
  if (!tflops) return FSLBM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSLBM_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) return FSLBM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  if (cudaMalloc(&out, 8) != cudaSuccess) return FSLBM_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  int rc = FSLBM_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == FSLBM_OK; ++rep) {  // the first run warms up
    cudaEventRecord(e0, st);
    k_dfma<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = FSLBM_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == FSLBM_OK) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return rc;
}
