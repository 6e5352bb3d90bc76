// FMA-throughput probe used for the FP64 / FP32 roofline denominators (include/gw_probe.h).
#include <cuda_runtime.h>

#include <string>

#include "../../include/gw_probe.h"
#include "internal.h"

namespace {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
cudaError_t time_chains(int blocks, int threads, int iters, double* tflops) {
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  for (int r = 0; r < 3; ++r) k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess) *tflops = 3.0 * 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return e;
}

}  // namespace

extern "C" gw_status gw_fp_peak(int device, double* fp64_tflops, double* fp32_tflops) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double t64 = 0, t32 = 0;
  if (e == cudaSuccess && fp64_tflops) e = time_chains<double>(sms * 4, 256, 1 << 13, &t64);
  if (e == cudaSuccess && fp32_tflops) e = time_chains<float>(sms * 4, 256, 1 << 15, &t32);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    gw::set_last_error(std::string("gw_fp_peak: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  if (fp64_tflops) *fp64_tflops = t64;
  if (fp32_tflops) *fp32_tflops = t32;
  return GW_OK;
}
