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
constexpr int kWTN = 64;     // output columns per residual block
constexpr int kWNmax = 384;  // largest N whose level sums stay exact in FP32
constexpr int kWStages = 4;  // shared-memory stages of the residual
constexpr uint32_t kWAChunk = kWSA * 2 * 128 * 16 * 2;  // bytes per (row block, K step): Re then Im digits
__host__ __device__ constexpr uint32_t wx_chunk(int SX) { return (uint32_t)SX * 2 * kWTN * 16 * 2; }
// dynamic shared memory of the residual: per stage the A digits s <= lmax of one
// component (128 x 16 each) and the SX digits of one component of X (kWTN x 16 each)
__host__ __device__ constexpr size_t w_residual_smem(int SX, int lmax) {
  return (size_t)kWStages * ((size_t)(lmax + 1) * 128 * 16 * 2 + (size_t)SX * kWTN * 16 * 2);
}

constexpr int kGJ32B = 32;    // panel width of the FP32 Gauss-Jordan inverse
constexpr int kGJ32C = 128;   // column chunk of its trailing update
// float2 elements of the multi-use buffer (pivot rows, exchange staging, row copies)
__host__ __device__ constexpr size_t gj32_buf_elems(int N) {
  return (size_t)2 * kGJ32B * kGJ32C > (size_t)16 * N ? (size_t)2 * kGJ32B * kGJ32C : (size_t)16 * N;
}
// dynamic shared memory of k_gj_inverse_f32
__host__ __device__ constexpr size_t gj32_smem(int N) {
  return ((size_t)N * kGJ32B + gj32_buf_elems(N)) * 8 + ((size_t)2 * N + 4 * kGJ32B) * 4;
}
__global__ void k_gj_inverse_f32(float2* __restrict__ A, int N, long long mat_stride, int* __restrict__ status);
__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, long long n);
__global__ void k_row_exponent(const double2* __restrict__ A, int* __restrict__ eA, int N, int batch);

__global__ void k_slice_A(const double2* __restrict__ A, const int* __restrict__ eA, uint16_t* __restrict__ Asl,
                          int N, long long n_total);
// Refinement products X R on the tensor cores: BF16x3 planes, 6 planes of 128 x 16 per
// (128-row block, 16-wide K step) chunk, kRefStages pipeline stages of 2 chunks.
constexpr uint32_t kRefChunk = 6 * 128 * 16 * 2;
constexpr int kRefStages = 4;
__host__ __device__ constexpr size_t w_refine_smem() { return (size_t)kRefStages * 2 * kRefChunk; }

// Scratch of one batch of tensor-core inverses (per matrix: three N^2 FP32 complex
// arrays, 2 kWSA and 2 kWSX1 BF16 digit planes and 6 BF16 term planes per element,
// 2 N exponents).
struct WtcBuffers {
  float2* X32;    // FP32 inverse X0 (the high part of X1)
  float2* lo;     // X1 - X0
  float2* R;      // residual I - A X (FP32)
  uint16_t* Asl;  // digits of A
  uint16_t* Xsl;  // digits of X, then the term planes of R
  uint16_t* PX;   // term planes of X0
  int* eA;
  int* eX;
  int* status;
};

// Raise the shared-memory limits of the kernels (once per device and size).
cudaError_t wtc_setup(size_t smem_gj32);

// ---- block Gauss-Jordan for N beyond kWNmax (kernels_wtc.cu) ----------------------
// Arguments of k_oz_panel_gemm: C = A B (accumulate 0) or C -= A B (1) from the digits
// of an M x K and a K x Nc panel (M a multiple of 128, Nc of kWTN, K of 16 and <= kWblkMaxK).
struct PanelGemmArgs {
  const uint16_t* Asl;
  const uint16_t* Bsl;
  const int* eA;
  const int* eB;
  double2* C;
  long long c_ms;  // matrix stride of C (elements)
  int ldc;         // row stride of C (elements)
  int M, Nc, K;
  int skip0, skip1;  // 128-row blocks of C left alone
  int accumulate;
  int* status;
};
// Scratch of one batch of block inverses of N x N with pivot blocks of bs (per matrix:
// the pivot block D, the row panel Rp, the digits of a bs-column and a bs-row panel, 2 N
// exponents) and the tensor-core inverse of the bs x bs pivot blocks.
struct WblkBuffers {
  double2* D;     // [batch][bs][bs]
  double2* Rp;    // [batch][bs][N]
  uint16_t* Asl;  // digits of the N x bs column panel (or of D)
  uint16_t* Bsl;  // digits of the bs x N row panel
  int* eA;        // [batch][N]
  int* eB;        // [batch][N]
  WtcBuffers inner;  // for batch matrices of bs x bs
};
// refinements of the FP32 inverse of each pivot block
constexpr int kWblkRefinements = 4;
// largest pivot block: the panel products keep one accumulator per level over both K
// halves, exact for levels 0..5 up to 256 complex terms
constexpr int kWblkMaxK = 256;
// Pivot block size for N (the largest multiple of 128 up to kWblkMaxK dividing N), or 0
// when N needs no blocks (N <= kWNmax) or has none (N not a multiple of 128).
int wblk_block_size(int N);
cudaError_t wblk_setup(size_t smem_gj32_bs);
// In place: mats[b] (FP64, N x N, Hermitian positive definite or with well-conditioned
// leading blocks) -> inverse, for b < batch; bs = wblk_block_size(N).
void wblk_inverse(const WblkBuffers& w, double2* mats, int batch, int N, int bs, size_t smem_gj32_bs,
                  cudaStream_t st);
// In place: mats[b] (FP64, N x N, N a multiple of 128) -> inverse, for b < batch, with
// `refinements` (at least 2) FP64-accurate refinements of the FP32 inverse.
void wtc_inverse(const WtcBuffers& w, double2* mats, int batch, int N, size_t smem_gj32, cudaStream_t st,
                 int refinements = 2);
__global__ void k_panel_col_exp(const double2* __restrict__ B, long long ms, int ld, int K, int Nc,
                                int* __restrict__ e);
__global__ void k_slice_panel_B(const double2* __restrict__ B, long long ms, int ld, const int* __restrict__ eB,
                                uint16_t* __restrict__ Bsl, int K, int Nc, long long n_thr);

}  // namespace gw
