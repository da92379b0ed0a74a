// gpe_peak.cu -- gp_fp_fma_rates: the measured FP64 and FP32 fused
// multiply-add rates of the current GPU (declared in include/gpe.h), the
// denominators of the ALU roofline the FP64 and double-float sweeps are held
// to (their memory traffic is far below the HBM bandwidth at these rates).
//
// Every thread runs kChains independent FMA chains of kIters steps (enough
// independent work to cover the pipe latency), on 8 blocks of 256 threads per
// SM; the result is written out so nothing is optimised away.  The rate is
// thread FMA instructions per second of the timed launch.
#include <cuda_runtime.h>

#include <string>

#include "gpe_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* out, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_rate(int blocks, double* rate) {
  T* out = nullptr;
  GP_CUDA(cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a in (0, 1) and b small: the chains stay finite
  fma_rate_kernel<T><<<blocks, 256>>>(out, (T)0.999, (T)1e-3);  // warm-up
  cudaEventRecord(e0);
  fma_rate_kernel<T><<<blocks, 256>>>(out, (T)0.999, (T)1e-3);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  gpe::count_launch(2);
  if (e != cudaSuccess) return gpe::fail(GP_ERR_CUDA, std::string("gp_fp_fma_rates: ") + cudaGetErrorString(e));
  *rate = (double)blocks * 256 * kChains * kIters / (ms * 1e-3);
  return GP_OK;
}

}  // namespace

extern "C" int gp_fp_fma_rates(double* dfma_per_s, double* ffma_per_s) {
  if (!dfma_per_s || !ffma_per_s) return gpe::fail(GP_ERR_INVALID, "gp_fp_fma_rates: NULL argument");
  int dev = 0, sms = 0;
  GP_CUDA(cudaGetDevice(&dev));
  GP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int rc = time_rate<double>(8 * sms, dfma_per_s);
  if (!rc) rc = time_rate<float>(64 * sms, ffma_per_s);
  return rc;
}
