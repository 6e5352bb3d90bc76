// Tensor-core W inverse: FP32 Gauss-Jordan + two refinements with an exactly sliced
// (BF16) residual on tcgen05.  Kernels in kernels_wtc.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gw {

constexpr int kWSA = 8;      // slices of the FP64 matrix (7 bits each)
constexpr int kWSX0 = 5;     // slices of the FP32 first inverse
constexpr int kWL0 = 5;      // first residual: products a_s x_t with s + t <= kWL0
constexpr int kWSX1 = 8;     // slices of the once-refined FP64 inverse
constexpr int kWLmax = 7;    // second residual: products a_s x_t with s + t <= kWLmax
constexpr int kWTN = 32;     // output columns per residual block
constexpr int kWNmax = 384;  // largest N whose level sums stay exact in FP32
constexpr uint32_t kWAChunk = kWSA * 2 * 128 * 16 * 2;  // bytes per (row block, K step)
// bytes of the A planes s <= lmax (the leading part of a chunk)
__host__ __device__ constexpr uint32_t wa_bytes(int lmax) {
  return (uint32_t)((lmax + 1 < kWSA ? lmax + 1 : kWSA) * 2 * 128 * 16 * 2);
}
__host__ __device__ constexpr uint32_t wx_chunk(int SX) { return (uint32_t)SX * 2 * kWTN * 16 * 2; }
__host__ __device__ constexpr size_t w_residual_smem(int SX, int lmax) {
  return 2 * (size_t)(wa_bytes(lmax) + wx_chunk(SX));
}

__global__ void k_gj_inverse_blocked_f32(float2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                                         int* status);
__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, long long n);
__global__ void k_row_exponent(const double2* __restrict__ A, int* __restrict__ eA, int N, int batch);

__global__ void k_slice_A(const double2* __restrict__ A, const int* __restrict__ eA, uint16_t* __restrict__ Asl,
                          int N, long long n_total);
// Scratch of one batch of tensor-core inverses (sizes per matrix: N^2 FP32 and three
// N^2 FP64 arrays, 2 kWSA and 2 kWSX1 BF16 slices per element, 2 N exponents, N pivots).
struct WtcBuffers {
  float2* X32;
  double2* X1;
  double2* R;
  uint16_t* Asl;
  uint16_t* Xsl;
  int* eA;
  int* eX;
  int* perm;
  int* status;
};

// Raise the shared-memory limits of the kernels (once per device and size).
cudaError_t wtc_setup(size_t smem_gj32);
// In place: mats[b] (FP64, N x N, N a multiple of 128) -> inverse, for b < batch.
void wtc_inverse(const WtcBuffers& w, double2* mats, int batch, int N, size_t smem_gj32, cudaStream_t st);

}  // namespace gw
