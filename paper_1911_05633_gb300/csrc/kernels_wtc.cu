// W solve on the tensor cores (Eq. W_1): each inverse (v(q)^-1, then (v^-1 - P)^-1) is
// computed in FP32 by Gauss-Jordan and refined twice, X <- X + X (I - A X), with the
// residual I - A X evaluated to FP64 accuracy on tcgen05 from exact BF16 slices of A
// and X (an Ozaki-type splitting): after a power-of-two scaling per row of A and per
// column of X, every entry is a sum of slices a_s = alpha_s 2^-7(s+1), |alpha_s| <= 128,
// each exact in BF16.  The products a_s x_t with s + t = L are multiples of 2^-7(L+2)
// whose sums over K = N <= 384 terms stay below 2^24 units in these accumulators:
// levels 0, 1, 2 (Re: ArXr - AiXi, Im: ArXi + AiXr together), level 3 (one product
// type per accumulator); levels >= 4 share one FP32 accumulator whose rounding stays
// at 2^-52 kappa of |A||X|.  The epilogue adds the levels in FP64.  Two refinements
// take the FP32 inverse (error ~ kappa 1e-7) to ~1e-12 for kappa ~ 2e3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "smem_limit.h"
#include "umma.h"
#include "wtc.h"

namespace gw {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

}  // namespace

// In-place FP32 Gauss-Jordan inverse, the FP32 form of k_gj_inverse_blocked.
__global__ void k_gj_inverse_blocked_f32(float2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                                     int* status) {
  extern __shared__ unsigned char smraw[];
  float2* Pan = reinterpret_cast<float2*>(smraw);  // [N][kGJB] panel columns
  float2* Prow = Pan + (size_t)N * kGJB;            // [kGJB][N] pivot rows (pre-update)
  float2* colk = Prow + (size_t)N * kGJB;           // [N]
  __shared__ float2 rowk[kGJB];
  __shared__ int pmk[kGJB];
  __shared__ float rv[32];
  __shared__ int ri[32];
  const int b = blockIdx.x;
  float2* M = A + (long long)b * mat_stride;
  int* pm = perm + (long long)b * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k0 = 0; k0 < N; k0 += kGJB) {
    const int bb = min(kGJB, N - k0);
    // load the panel
    for (int x = tid; x < N * bb; x += nt) {
      const int i = x / bb, m = x - (x / bb) * bb;
      Pan[i * kGJB + m] = M[(long long)i * N + k0 + m];
    }
    __syncthreads();
    for (int m = 0; m < bb; ++m) {
      const int k = k0 + m;
      float best = -1.0f;
      int bi = k;
      for (int i = k + tid; i < N; i += nt) {
        const float2 z = Pan[i * kGJB + m];
        const float a = fabsf(z.x) + fabsf(z.y);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
      __syncthreads();
      if (wid == 0) {
        best = (lane < nw) ? rv[lane] : -1.0f;
        bi = (lane < nw) ? ri[lane] : N;
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          ri[0] = bi;
          pm[k] = bi;
          pmk[m] = bi;
          if (!(best > 0.0f)) atomicExch(status, 1);
        }
      }
      __syncthreads();
      const int p = ri[0];
      if (p != k && tid < bb) {
        const float2 t = Pan[k * kGJB + tid];
        Pan[k * kGJB + tid] = Pan[p * kGJB + tid];
        Pan[p * kGJB + tid] = t;
      }
      __syncthreads();
      const float2 d = Pan[k * kGJB + m];
      const float den = d.x * d.x + d.y * d.y;
      const float2 inv = (den > 0.0f) ? make_float2(d.x / den, -d.y / den) : make_float2(0.0f, 0.0f);
      for (int i = tid; i < N; i += nt) colk[i] = (i == k) ? make_float2(0.0f, 0.0f) : Pan[i * kGJB + m];
      if (tid < bb) rowk[tid] = (tid == m) ? inv : cmul(Pan[k * kGJB + tid], inv);
      __syncthreads();
      for (int x = tid; x < N * bb; x += nt) {
        const int i = x / bb, j = x - (x / bb) * bb;
        if (i == k) {
          Pan[i * kGJB + j] = rowk[j];
        } else {
          const float2 f = colk[i];
          const float2 z = (j == m) ? make_float2(0.0f, 0.0f) : Pan[i * kGJB + j];
          Pan[i * kGJB + j] = cfma(make_float2(-f.x, -f.y), rowk[j], z);
        }
      }
      __syncthreads();
    }
    // row exchanges on the other columns, then the pivot rows (pre-update) to shared memory
    for (int j = tid; j < N; j += nt) {
      if (j >= k0 && j < k0 + bb) continue;
      for (int m = 0; m < bb; ++m) {
        const int k = k0 + m, p = pmk[m];
        if (p != k) {
          const float2 t = M[(long long)k * N + j];
          M[(long long)k * N + j] = M[(long long)p * N + j];
          M[(long long)p * N + j] = t;
        }
      }
      for (int m = 0; m < bb; ++m) Prow[m * N + j] = M[(long long)(k0 + m) * N + j];
    }
    __syncthreads();
    // A[:, T] += (Pan - I[:, panel]) Prow   (one warp per row, lanes along j)
    for (int i = wid; i < N; i += nw) {
      float2 z[kGJB];
#pragma unroll
      for (int m = 0; m < kGJB; ++m) {
        z[m] = (m < bb) ? Pan[i * kGJB + m] : make_float2(0.0f, 0.0f);
        if (i == k0 + m) z[m].x -= 1.0f;
      }
      float2* Mi = M + (long long)i * N;
      for (int j = lane; j < N; j += 32) {
        if (j >= k0 && j < k0 + bb) continue;
        float2 acc = Mi[j];
#pragma unroll
        for (int m = 0; m < kGJB; ++m)
          if (m < bb) acc = cfma(z[m], Prow[m * N + j], acc);
        Mi[j] = acc;
      }
    }
    // the panel itself
    for (int x = tid; x < N * bb; x += nt) {
      const int i = x / bb, m = x - (x / bb) * bb;
      M[(long long)i * N + k0 + m] = Pan[i * kGJB + m];
    }
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    const int p = pm[k];
    if (p != k) {
      for (int i = tid; i < N; i += nt) {
        const float2 t = M[(long long)i * N + k];
        M[(long long)i * N + k] = M[(long long)i * N + p];
        M[(long long)i * N + p] = t;
      }
    }
    __syncthreads();
  }
}

namespace {

using namespace umma;

constexpr uint64_t kWaitNs = 500ull * 1000ull * 1000ull;

__device__ __forceinline__ uint16_t bf16_bits(double v) {
  // v is exactly representable in BF16 (<= 8 significant bits): take the top half of its FP32 form
  const float f = (float)v;
  return (uint16_t)(__float_as_uint(f) >> 16);
}

// scale exponent e with max |x| < 2^e (0 for an all-zero row / column)
__device__ __forceinline__ int scale_exponent(double m) { return m > 0.0 ? ilogb(m) + 1 : 0; }

}  // namespace

__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, long long n) {
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double2 z = src[x];
    dst[x] = make_float2((float)z.x, (float)z.y);
  }
}

// one warp per row: eA[b][i] with max_k max(|Re|, |Im|) A[b][i][k] < 2^eA
__global__ void k_row_exponent(const double2* __restrict__ A, int* __restrict__ eA, int N, int batch) {
  const int warps = blockDim.x >> 5;
  const long long row = (long long)blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= (long long)batch * N) return;
  const double2* a = A + row * N;
  double m = 0.0;
  for (int k = lane; k < N; k += 32) m = fmax(m, fmax(fabs(a[k].x), fabs(a[k].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) eA[row] = scale_exponent(m);
}

// one thread per column j: eX[b][j] with max_k max(|Re|, |Im|) X[b][k][j] < 2^eX
template <typename T>
__global__ void k_col_exponent(const T* __restrict__ X, int* __restrict__ eX, int N) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const T* x = X + (long long)b * N * N;
  double m = 0.0;
  for (int k = 0; k < N; ++k) m = fmax(m, fmax(fabs((double)x[(long long)k * N + j].x), fabs((double)x[(long long)k * N + j].y)));
  eX[(long long)b * N + j] = scale_exponent(m);
}

// A operand slices: element (i, k) of matrix b -> kWSA slices of Re and Im in the
// K-major tile layout, one contiguous chunk per (matrix, 128-row block, 16-column step).
__global__ void k_slice_A(const double2* __restrict__ A, const int* __restrict__ eA, uint16_t* __restrict__ Asl,
                          int N, long long n_total) {
  const int NKS = N / 16, NIB = N / 128;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_total; x += (long long)gridDim.x * blockDim.x) {
    const long long b = x / ((long long)N * N);
    const int r = (int)(x - b * N * N);
    const int i = r / N, k = r - (r / N) * N;
    const double2 z = A[x];
    const int e = eA[b * N + i];
    const long long chunk = ((b * NIB + i / 128) * NKS + k / 16) * (long long)(kWAChunk / 2);
    const uint32_t off = kmajor_offset(128, i & 127, k & 15) / 2;
    double v[2] = {ldexp(z.x, -e), ldexp(z.y, -e)};
    for (int c = 0; c < 2; ++c) {
      double rres = v[c];
      for (int s = 0; s < kWSA; ++s) {
        const double sc = ldexp(1.0, 7 * (s + 1));
        const double a = rint(rres * sc) / sc;  // alpha_s 2^-7(s+1)
        rres -= a;
        Asl[chunk + (long long)(s * 2 + c) * (128 * 16) + off] = bf16_bits(a);
      }
    }
  }
}

// X operand slices: element X[k][j] of matrix b (k = reduction index) -> SX slices of
// Re and Im in the K-major layout of the B operand (rows j), one chunk per (matrix,
// kWTN-column block, 16-row step).
template <typename T, int SX>
__global__ void k_slice_X(const T* __restrict__ X, const int* __restrict__ eX, uint16_t* __restrict__ Xsl, int N,
                          long long n_total) {
  const int NKS = N / 16, NJB = N / kWTN;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_total; x += (long long)gridDim.x * blockDim.x) {
    const long long b = x / ((long long)N * N);
    const int r = (int)(x - b * N * N);
    const int k = r / N, j = r - (r / N) * N;
    const T z = X[x];
    const int e = eX[b * N + j];
    const long long chunk = ((b * NJB + j / kWTN) * NKS + k / 16) * (long long)(wx_chunk(SX) / 2);
    const uint32_t off = kmajor_offset(kWTN, j % kWTN, k & 15) / 2;
    double v[2] = {ldexp((double)z.x, -e), ldexp((double)z.y, -e)};
    for (int c = 0; c < 2; ++c) {
      double rres = v[c];
      for (int t = 0; t < SX; ++t) {
        const double sc = ldexp(1.0, 7 * (t + 1));
        const double a = rint(rres * sc) / sc;
        rres -= a;
        Xsl[chunk + (long long)(t * 2 + c) * (kWTN * 16) + off] = bf16_bits(a);
      }
    }
  }
}

// R[b] = I - A[b] X[b] for one 128 x kWTN output tile per block (128 threads).  Twelve
// FP32 accumulators of kWTN columns in tensor memory: for Re and Im, the levels 0, 1, 2
// (both product types), level 3 (one accumulator per product type) and levels >= 4.
template <int SX>
__global__ void __launch_bounds__(128, 1)
k_ozaki_residual(const uint16_t* __restrict__ Asl, const uint16_t* __restrict__ Xsl, const int* __restrict__ eA,
                 const int* __restrict__ eX, double2* __restrict__ R, int N, int* status) {
  constexpr uint32_t XC = wx_chunk(SX);
  constexpr uint32_t PX = kWTN * 16 * 2;  // bytes per X plane
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[2];
  __shared__ __align__(8) uint64_t mmad[2];
  const int jb = blockIdx.x, ib = blockIdx.y;
  const long long b = blockIdx.z;
  const int NKS = N / 16, NIB = N / 128, NJB = N / kWTN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&mmad[0], 1);
    mbar_init(&mmad[1], 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const unsigned char* Abase = reinterpret_cast<const unsigned char*>(Asl) + ((b * NIB + ib) * NKS) * (long long)kWAChunk;
  const unsigned char* Xbase = reinterpret_cast<const unsigned char*>(Xsl) + ((b * NJB + jb) * NKS) * (long long)XC;
  unsigned char* stage[2] = {sm, sm + kWAChunk + XC};
  bool ok = true;
  if (tid == 0) {
    const uint32_t id = idesc_bf16_f32(128, kWTN), idn = idesc_bf16_f32_negA(128, kWTN);
    for (int s = 0; s < 2 && s < NKS; ++s) {
      mbar_arrive_expect_tx(&full[s], kWAChunk + XC);
      bulk_g2s(stage[s], Abase + (long long)s * kWAChunk, kWAChunk, &full[s]);
      bulk_g2s(stage[s] + kWAChunk, Xbase + (long long)s * XC, XC, &full[s]);
    }
    uint32_t used = 0;  // accumulator initialised (bit per accumulator)
    for (int ks = 0; ks < NKS && ok; ++ks) {
      const int st = ks & 1;
      const uint32_t par = (uint32_t)(ks >> 1) & 1u;
      if (!mbar_wait(&full[st], par, kWaitNs, status)) { ok = false; break; }
      fence_after_sync();
      const uint32_t aB = smem_u32(stage[st]), xB = aB + kWAChunk;
      for (int t = 0; t < SX; ++t) {
        for (int s = 0; s < kWSA && s + t <= kWLmax; ++s) {
          const int L = s + t;
          // accumulators (columns q * kWTN): Re 0..5, Im 6..11
          int r1, r2, i1, i2;
          if (L <= 2) { r1 = r2 = L; i1 = i2 = 6 + L; }
          else if (L == 3) { r1 = 3; r2 = 4; i1 = 9; i2 = 10; }
          else { r1 = r2 = 5; i1 = i2 = 11; }
          const uint64_t dar = smem_desc(aB + (uint32_t)(s * 2 + 0) * 4096u, 128, 256);
          const uint64_t dai = smem_desc(aB + (uint32_t)(s * 2 + 1) * 4096u, 128, 256);
          const uint64_t dxr = smem_desc(xB + (uint32_t)(t * 2 + 0) * PX, 128, 256);
          const uint64_t dxi = smem_desc(xB + (uint32_t)(t * 2 + 1) * PX, 128, 256);
          // Re += Ar Xr - Ai Xi ; Im += Ar Xi + Ai Xr
          mma_bf16(tm + (uint32_t)r1 * kWTN, dar, dxr, id, (used >> r1) & 1u);
          used |= 1u << r1;
          mma_bf16(tm + (uint32_t)r2 * kWTN, dai, dxi, idn, (used >> r2) & 1u);
          used |= 1u << r2;
          mma_bf16(tm + (uint32_t)i1 * kWTN, dar, dxi, id, (used >> i1) & 1u);
          used |= 1u << i1;
          mma_bf16(tm + (uint32_t)i2 * kWTN, dai, dxr, id, (used >> i2) & 1u);
          used |= 1u << i2;
        }
      }
      mma_commit(&mmad[st]);
      if (ks + 2 < NKS) {
        // refill this stage once its products are done
        if (!mbar_wait(&mmad[st], par, kWaitNs, status)) { ok = false; break; }
        mbar_arrive_expect_tx(&full[st], kWAChunk + XC);
        bulk_g2s(stage[st], Abase + (long long)(ks + 2) * kWAChunk, kWAChunk, &full[st]);
        bulk_g2s(stage[st] + kWAChunk, Xbase + (long long)(ks + 2) * XC, XC, &full[st]);
      }
    }
  }
  // every thread waits for the last products; one verdict for the block
  const int last = NKS - 1;
  const bool done = ok && mbar_wait(&mmad[last & 1], (uint32_t)(last >> 1) & 1u, kWaitNs, status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 2);
  } else {
    const int r = 32 * warp + lane;
    const int i = ib * 128 + r;
    const int ea = eA[b * N + i];
    double2* Ro = R + (b * N + i) * (long long)N;
    for (int c0 = 0; c0 < kWTN; c0 += 16) {
      float v[12][16];
#pragma unroll
      for (int q = 0; q < 12; ++q) tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)(q * kWTN + c0), v[q]);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = jb * kWTN + c0 + c;
        const double sc = ldexp(1.0, ea + eX[b * N + j]);
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int q = 5; q >= 0; --q) re += (double)v[q][c];
#pragma unroll
        for (int q = 11; q >= 6; --q) im += (double)v[q][c];
        Ro[j] = make_double2((i == j ? 1.0 : 0.0) - sc * re, -sc * im);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// X1[b] = X0[b] + X0[b] R[b] with the product in FP32 arithmetic (R is small), written as
// FP64.  64 x 64 output tile per block, 256 threads, 4 x 4 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256)
k_refine_update(const T* __restrict__ X0, const double2* __restrict__ R, double2* __restrict__ X1, int N) {
  __shared__ float2 Xs[16][64 + 1];
  __shared__ float2 Rs[16][64 + 1];
  const long long b = blockIdx.z;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const T* X = X0 + b * (long long)N * N;
  const double2* Rb = R + b * (long long)N * N;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[u][w] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < N; k0 += 16) {
    for (int x = threadIdx.x; x < 64 * 16; x += 256) {
      const int r = x / 16, c = x - (x / 16) * 16;  // X tile: rows i0 + r, cols k0 + c
      const T xv = X[(long long)(i0 + r) * N + k0 + c];
      Xs[c][r] = make_float2((float)xv.x, (float)xv.y);
      const int r2 = x / 64, c2 = x - (x / 64) * 64;  // R tile: rows k0 + r2, cols j0 + c2
      const double2 z = Rb[(long long)(k0 + r2) * N + j0 + c2];
      Rs[r2][c2] = make_float2((float)z.x, (float)z.y);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      float2 a[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Xs[k][ty + 16 * u];
#pragma unroll
      for (int w = 0; w < 4; ++w) bb[w] = Rs[k][tx + 16 * w];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = cfma(a[u], bb[w], acc[u][w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const long long o = b * (long long)N * N + (long long)(i0 + ty + 16 * u) * N + j0 + tx + 16 * w;
      const T x0 = X0[o];
      X1[o] = make_double2((double)x0.x + (double)acc[u][w].x, (double)x0.y + (double)acc[u][w].y);
    }
}

cudaError_t wtc_setup(size_t smem_gj32) {
  cudaError_t e = raise_smem_limit(k_gj_inverse_blocked_f32, smem_gj32);
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX0>, w_residual_smem(kWSX0));
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX1>, w_residual_smem(kWSX1));
  return e;
}

void wtc_inverse(const WtcBuffers& w, double2* mats, int batch, int N, size_t smem_gj32, cudaStream_t st) {
  const long long NN = (long long)N * N;
  const long long tot = (long long)batch * NN;
  const unsigned g1 = (unsigned)((tot + 255) / 256 < 65535LL * 8 ? (tot + 255) / 256 : 65535LL * 8);
  const dim3 gcol((unsigned)((N + 127) / 128), (unsigned)batch);
  const dim3 gres((unsigned)(N / kWTN), (unsigned)(N / 128), (unsigned)batch);
  const dim3 gupd((unsigned)(N / 64), (unsigned)(N / 64), (unsigned)batch);
  // X0: FP32 Gauss-Jordan
  k_to_f32<<<g1, 256, 0, st>>>(mats, w.X32, tot);
  k_gj_inverse_blocked_f32<<<batch, 512, smem_gj32, st>>>(w.X32, w.perm, N, NN, w.status);
  // slices of A (kept for both residuals)
  k_row_exponent<<<(unsigned)((batch * (long long)N + 7) / 8), 256, 0, st>>>(mats, w.eA, N, batch);
  k_slice_A<<<g1, 256, 0, st>>>(mats, w.eA, w.Asl, N, tot);
  // X1 = X0 + X0 (I - A X0)
  k_col_exponent<float2><<<gcol, 128, 0, st>>>(w.X32, w.eX, N);
  k_slice_X<float2, kWSX0><<<g1, 256, 0, st>>>(w.X32, w.eX, w.Xsl, N, tot);
  k_ozaki_residual<kWSX0><<<gres, 128, w_residual_smem(kWSX0), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R, N, w.status);
  k_refine_update<float2><<<gupd, 256, 0, st>>>(w.X32, w.R, w.X1, N);
  // X2 = X1 + X1 (I - A X1), written over A
  k_col_exponent<double2><<<gcol, 128, 0, st>>>(w.X1, w.eX, N);
  k_slice_X<double2, kWSX1><<<g1, 256, 0, st>>>(w.X1, w.eX, w.Xsl, N, tot);
  k_ozaki_residual<kWSX1><<<gres, 128, w_residual_smem(kWSX1), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R, N, w.status);
  k_refine_update<double2><<<gupd, 256, 0, st>>>(w.X1, w.R, mats, N);
}

}  // namespace gw
