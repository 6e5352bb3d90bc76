// W solve on the tensor cores (Eq. W_1): each inverse (v(q)^-1, then (v^-1 - P)^-1) is
// computed in FP32 by Gauss-Jordan and refined twice, X <- X + X (I - A X), with the
// residual I - A X evaluated to FP64 accuracy on tcgen05 from exact BF16 slices of A
// and X (an Ozaki-type splitting): after a power-of-two scaling per row of A and per
// column of X, every entry is a sum of slices a_s = alpha_s 2^-7(s+1), |alpha_s| <= 128,
// each exact in BF16.  The products a_s x_t with s + t = L are multiples of 2^-7(L+2).
// For K = N <= 384 terms their sums stay below 2^24 such units in these accumulators,
// so FP32 accumulation is exact: levels 0, 1, 2 (Re: ArXr - AiXi, Im: ArXi + AiXr
// together), levels 3 and 4 (one product type per accumulator).  The levels >= 5 share
// one FP32 accumulator, whose rounding is ~2^-60 N of |A||X|.  The epilogue adds the
// levels in FP64, level 0 first against the identity.  Two refinements take the FP32
// inverse (error ~ kappa 1e-7) to ~1e-13 for kappa ~ 2e3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "smem_limit.h"
#include "umma.h"
#include "wtc.h"
#include "ktimer.h"

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

// Signed base-2^7 digits of one scaled entry: m = round(v 2^56) for |v| < 1, then
// digit s = round(m / 2^(49 - 7 s)) taken from the top, so that v = sum_s d_s 2^-7(s+1)
// up to 2^-57 with |d_0| <= 128 and |d_s| <= 64 after it; every d_s 2^-7(s+1) is exact
// in BF16 (at most 8 significant bits).  Integer arithmetic only after one FP64 scaling.
__device__ __forceinline__ long long fixed56(double x, int e) {
  // x 2^(56 - e) with |x| < 2^e; the power of two is built from its exponent bits
  const double p = __longlong_as_double((long long)(1023 + 56 - e) << 52);
  return __double2ll_rn(x * p);
}
__device__ __forceinline__ int next_digit(long long& m, int s) {
  const int sh = 49 - 7 * s;
  const long long d = sh > 0 ? (m + (1ll << (sh - 1))) >> sh : m;
  m -= d << sh;
  return (int)d;
}
// bits of d 2^-7(s+1) in BF16 (exact)
__device__ __forceinline__ uint32_t digit_bf16(int d, int s) {
  const float sc = __int_as_float((127 - 7 * (s + 1)) << 23);
  return __float_as_uint((float)d * sc) >> 16;
}

// A operand slices.  Element (i, k) of matrix b -> kWSA digits of Re and Im in the
// K-major tile layout, one contiguous chunk per (matrix, 128-row block, 16-column step)
// holding 2 kWSA planes of 128 x 16.  One thread per (row i, 8 consecutive k): it reads
// 128 contiguous bytes and writes one 16-byte row of a core matrix per plane; the 32
// lanes of a warp (i % 8, k half, (i / 8) % 2) fill 512 contiguous bytes of each plane.
__global__ void k_slice_A(const double2* __restrict__ A, const int* __restrict__ eA, uint16_t* __restrict__ Asl,
                          int N, long long n_total) {
  const int NKS = N / 16, NIB = N / 128;
  const long long n_thr = n_total / 8;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;  // (b, ib, ks, row group pair)
    const int gp = (int)(w % 8); w /= 8;
    const int ks = (int)(w % NKS); w /= NKS;
    const int ib = (int)(w % NIB);
    const long long b = w / NIB;
    const int h = (lane >> 3) & 1;
    const int il = (lane & 7) + 8 * ((lane >> 4) + 2 * gp);  // row within the 128-row block
    const int i = ib * 128 + il;
    const int k0 = ks * 16 + 8 * h;
    const int e = eA[b * N + i];
    const double2* src = A + (b * N + i) * (long long)N + k0;
    long long mr[8], mi[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 z = src[u];
      mr[u] = fixed56(z.x, e);
      mi[u] = fixed56(z.y, e);
    }
    uint16_t* chunk = Asl + ((b * NIB + ib) * NKS + ks) * (long long)(kWAChunk / 2);
    const uint32_t off = kmajor_offset(128, il, 8 * h) / 2;
#pragma unroll
    for (int s = 0; s < kWSA; ++s) {
      uint32_t pr[4], pi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t r0 = digit_bf16(next_digit(mr[2 * u], s), s), r1 = digit_bf16(next_digit(mr[2 * u + 1], s), s);
        const uint32_t i0 = digit_bf16(next_digit(mi[2 * u], s), s), i1 = digit_bf16(next_digit(mi[2 * u + 1], s), s);
        pr[u] = r0 | (r1 << 16);
        pi[u] = i0 | (i1 << 16);
      }
      *reinterpret_cast<uint4*>(chunk + (s * 2 + 0) * (128 * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (s * 2 + 1) * (128 * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// X operand slices.  Element X[k][j] of matrix b (k = reduction index) -> SX digits of
// Re and Im in the K-major layout of the B operand (rows j), one chunk per (matrix,
// kWTN-column block, 16-row step).  One thread per (column j, 8 consecutive k); lanes
// (j % 8, k half, (j / 8) % 2) read 128-byte row segments and fill 512 contiguous bytes
// of each plane.
template <typename T, int SX>
__global__ void k_slice_X(const T* __restrict__ X, const int* __restrict__ eX, uint16_t* __restrict__ Xsl, int N,
                          long long n_total) {
  static_assert(kWTN == 32, "two 16-column halves per column block");
  const int NKS = N / 16, NJB = N / kWTN;
  const long long n_thr = n_total / 8;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;  // (b, jb, ks, column half)
    const int jh = (int)(w & 1); w >>= 1;
    const int ks = (int)(w % NKS); w /= NKS;
    const int jb = (int)(w % NJB);
    const long long b = w / NJB;
    const int h = (lane >> 3) & 1;
    const int jl = (lane & 7) + 8 * ((lane >> 4) + 2 * jh);  // column within the block
    const int j = jb * kWTN + jl;
    const int k0 = ks * 16 + 8 * h;
    const int e = eX[b * N + j];
    const T* src = X + (b * N + k0) * (long long)N + j;
    long long mr[8], mi[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T z = src[(long long)u * N];
      mr[u] = fixed56((double)z.x, e);
      mi[u] = fixed56((double)z.y, e);
    }
    uint16_t* chunk = Xsl + ((b * NJB + jb) * NKS + ks) * (long long)(wx_chunk(SX) / 2);
    const uint32_t off = kmajor_offset(kWTN, jl, 8 * h) / 2;
#pragma unroll
    for (int t = 0; t < SX; ++t) {
      uint32_t pr[4], pi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t r0 = digit_bf16(next_digit(mr[2 * u], t), t), r1 = digit_bf16(next_digit(mr[2 * u + 1], t), t);
        const uint32_t i0 = digit_bf16(next_digit(mi[2 * u], t), t), i1 = digit_bf16(next_digit(mi[2 * u + 1], t), t);
        pr[u] = r0 | (r1 << 16);
        pi[u] = i0 | (i1 << 16);
      }
      *reinterpret_cast<uint4*>(chunk + (t * 2 + 0) * (kWTN * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (t * 2 + 1) * (kWTN * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// Accumulator (columns q kWTN) of the products a_s x_t, s + t = L: Re 0..7, Im 8..15;
// `neg` selects Ai Xi (subtracted from Re), `imag` the Im products.
__host__ __device__ constexpr int ozaki_bucket(int L, bool second_type, bool imag) {
  return (imag ? 8 : 0) + (L <= 2 ? L : L == 3 ? (second_type ? 4 : 3) : L == 4 ? (second_type ? 6 : 5) : 7);
}

// The 4 x (number of (s, t) pairs) MMAs of one 16-wide K step.  Fully unrolled, so the
// accumulator indices, shared-memory offsets and first-use flags are constants.
template <int SX, int LMAX, bool FIRST>
__device__ __forceinline__ void ozaki_issue_step(uint32_t tm, uint64_t da0, uint64_t dx0, uint32_t id, uint32_t idn) {
  constexpr uint32_t PA = 128 * 16 * 2, PX = kWTN * 16 * 2;  // bytes per A / X plane
  uint32_t used = 0;
#pragma unroll
  for (int t = 0; t < SX; ++t) {
#pragma unroll
    for (int s = 0; s < kWSA; ++s) {
      if (s + t <= LMAX) {
        const int L = s + t;
        const int r1 = ozaki_bucket(L, false, false), r2 = ozaki_bucket(L, true, false);
        const int i1 = ozaki_bucket(L, false, true), i2 = ozaki_bucket(L, true, true);
        // descriptor start addresses are in 16-byte units in the low bits
        const uint64_t dar = da0 + (uint64_t)(((s * 2 + 0) * PA) >> 4);
        const uint64_t dai = da0 + (uint64_t)(((s * 2 + 1) * PA) >> 4);
        const uint64_t dxr = dx0 + (uint64_t)(((t * 2 + 0) * PX) >> 4);
        const uint64_t dxi = dx0 + (uint64_t)(((t * 2 + 1) * PX) >> 4);
        // Re += Ar Xr - Ai Xi ; Im += Ar Xi + Ai Xr
        mma_bf16(tm + (uint32_t)r1 * kWTN, dar, dxr, id, FIRST ? (used >> r1) & 1u : 1u);
        used |= 1u << r1;
        mma_bf16(tm + (uint32_t)r2 * kWTN, dai, dxi, idn, FIRST ? (used >> r2) & 1u : 1u);
        used |= 1u << r2;
        mma_bf16(tm + (uint32_t)i1 * kWTN, dar, dxi, id, FIRST ? (used >> i1) & 1u : 1u);
        used |= 1u << i1;
        mma_bf16(tm + (uint32_t)i2 * kWTN, dai, dxr, id, FIRST ? (used >> i2) & 1u : 1u);
        used |= 1u << i2;
      }
    }
  }
}

// R[b] = I - A[b] X[b] for one 128 x kWTN output tile per block (128 threads), from the
// A slices s <= LMAX and SX slices of X, products with s + t <= LMAX.  Sixteen FP32
// accumulators of kWTN columns fill the 512 tensor-memory columns: for Re and Im, the
// levels 0, 1, 2 (both product types together), levels 3 and 4 (one accumulator per
// product type) and the levels >= 5.  Two shared-memory stages: while the products of
// K step ks run, the stage of step ks - 1 is refilled with step ks + 1.
template <int SX, int LMAX>
__global__ void __launch_bounds__(128, 1)
k_ozaki_residual(const uint16_t* __restrict__ Asl, const uint16_t* __restrict__ Xsl, const int* __restrict__ eA,
                 const int* __restrict__ eX, double2* __restrict__ R, int N, int* status) {
  static_assert(LMAX >= 5 && LMAX < kWSA, "every accumulator receives a product; A has kWSA slices");
  constexpr uint32_t XC = wx_chunk(SX);
  constexpr uint32_t AC = wa_bytes(LMAX);  // the leading planes s <= LMAX of each A chunk
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
  unsigned char* const stage0 = sm;
  unsigned char* const stage1 = sm + AC + XC;
  bool ok = true;
  if (tid == 0) {
    const uint32_t id = idesc_bf16_f32(128, kWTN), idn = idesc_bf16_f32_negA(128, kWTN);
    const uint64_t da0 = smem_desc(smem_u32(stage0), 128, 256), da1 = smem_desc(smem_u32(stage1), 128, 256);
    const uint64_t dx0 = smem_desc(smem_u32(stage0) + AC, 128, 256), dx1 = smem_desc(smem_u32(stage1) + AC, 128, 256);
    for (int s = 0; s < 2 && s < NKS; ++s) {
      unsigned char* const dst = s ? stage1 : stage0;
      mbar_arrive_expect_tx(&full[s], AC + XC);
      bulk_g2s(dst, Abase + (long long)s * kWAChunk, AC, &full[s]);
      bulk_g2s(dst + AC, Xbase + (long long)s * XC, XC, &full[s]);
    }
    for (int ks = 0; ks < NKS; ++ks) {
      const int st = ks & 1;
      if (!mbar_wait(&full[st], (uint32_t)(ks >> 1) & 1u, kWaitNs, status)) { ok = false; break; }
      fence_after_sync();
      const uint64_t da = st ? da1 : da0, dx = st ? dx1 : dx0;
      if (ks == 0) ozaki_issue_step<SX, LMAX, true>(tm, da, dx, id, idn);
      else ozaki_issue_step<SX, LMAX, false>(tm, da, dx, id, idn);
      mma_commit(&mmad[st]);
      if (ks >= 1 && ks + 1 < NKS) {
        // the products of step ks - 1 are done once its commit arrives: refill its stage
        const int so = st ^ 1;
        if (!mbar_wait(&mmad[so], (uint32_t)((ks - 1) >> 1) & 1u, kWaitNs, status)) { ok = false; break; }
        unsigned char* const dst = so ? stage1 : stage0;
        mbar_arrive_expect_tx(&full[so], AC + XC);
        bulk_g2s(dst, Abase + (long long)(ks + 1) * kWAChunk, AC, &full[so]);
        bulk_g2s(dst + AC, Xbase + (long long)(ks + 1) * XC, XC, &full[so]);
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
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int c0 = 0; c0 < kWTN; c0 += 16) {
      // level 0 exactly against the identity, then the smaller levels added from the bottom
      double re[16], im[16];
      float v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) { re[c] = 0.0; im[c] = 0.0; }
#pragma unroll 1
      for (int q = 7; q >= 1; --q) {
        tmem_ld16(tm + lane_base + (uint32_t)(q * kWTN + c0), v);
#pragma unroll
        for (int c = 0; c < 16; ++c) re[c] += (double)v[c];
        tmem_ld16(tm + lane_base + (uint32_t)((8 + q) * kWTN + c0), v);
#pragma unroll
        for (int c = 0; c < 16; ++c) im[c] += (double)v[c];
      }
      float v0r[16], v0i[16];
      tmem_ld16(tm + lane_base + (uint32_t)c0, v0r);
      tmem_ld16(tm + lane_base + (uint32_t)(8 * kWTN + c0), v0i);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = jb * kWTN + c0 + c;
        const double sc = ldexp(1.0, ea + eX[b * N + j]);
        const double r0 = (i == j ? 1.0 : 0.0) - sc * (double)v0r[c];
        const double i0 = -sc * (double)v0i[c];
        Ro[j] = make_double2(r0 - sc * re[c], i0 - sc * im[c]);
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
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX0, kWL0>, w_residual_smem(kWSX0, kWL0));
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX1, kWLmax>, w_residual_smem(kWSX1, kWLmax));
  return e;
}

void wtc_inverse(const WtcBuffers& w, double2* mats, int batch, int N, size_t smem_gj32, cudaStream_t st) {
  const long long NN = (long long)N * N;
  const long long tot = (long long)batch * NN;
  const unsigned g1 = (unsigned)((tot + 255) / 256 < 65535LL * 8 ? (tot + 255) / 256 : 65535LL * 8);
  const long long t8 = tot / 8;  // slicing threads: one per 8 consecutive elements
  const unsigned g8 = (unsigned)((t8 + 255) / 256 < 65535LL * 8 ? (t8 + 255) / 256 : 65535LL * 8);
  const dim3 gcol((unsigned)((N + 127) / 128), (unsigned)batch);
  const dim3 gres((unsigned)(N / kWTN), (unsigned)(N / 128), (unsigned)batch);
  const dim3 gupd((unsigned)(N / 64), (unsigned)(N / 64), (unsigned)batch);
  // X0: FP32 Gauss-Jordan
  {
    gw::TimedLaunch tl_("k_to_f32", st);
    k_to_f32<<<g1, 256, 0, st>>>(mats, w.X32, tot);
  }
  {
    gw::TimedLaunch tl_("k_gj_inverse_blocked_f32", st);
    k_gj_inverse_blocked_f32<<<batch, 512, smem_gj32, st>>>(w.X32, w.perm, N, NN, w.status);
  }
  // slices of A (kept for both residuals)
  {
    gw::TimedLaunch tl_("k_row_exponent", st);
    k_row_exponent<<<(unsigned)((batch * (long long)N + 7) / 8), 256, 0, st>>>(mats, w.eA, N, batch);
  }
  {
    gw::TimedLaunch tl_("k_slice_A", st);
    k_slice_A<<<g8, 256, 0, st>>>(mats, w.eA, w.Asl, N, tot);
  }
  // X1 = X0 + X0 (I - A X0)
  {
    gw::TimedLaunch tl_("k_col_exponent", st);
    k_col_exponent<float2><<<gcol, 128, 0, st>>>(w.X32, w.eX, N);
  }
  {
    gw::TimedLaunch tl_("k_slice_X<float2>", st);
    k_slice_X<float2, kWSX0><<<g8, 256, 0, st>>>(w.X32, w.eX, w.Xsl, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_ozaki_residual<first>", st);
    k_ozaki_residual<kWSX0, kWL0><<<gres, 128, w_residual_smem(kWSX0, kWL0), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R, N,
                                                                                  w.status);
  }
  {
    gw::TimedLaunch tl_("k_refine_update<float2>", st);
    k_refine_update<float2><<<gupd, 256, 0, st>>>(w.X32, w.R, w.X1, N);
  }
  // X2 = X1 + X1 (I - A X1), written over A
  {
    gw::TimedLaunch tl_("k_col_exponent", st);
    k_col_exponent<double2><<<gcol, 128, 0, st>>>(w.X1, w.eX, N);
  }
  {
    gw::TimedLaunch tl_("k_slice_X<double2>", st);
    k_slice_X<double2, kWSX1><<<g8, 256, 0, st>>>(w.X1, w.eX, w.Xsl, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_ozaki_residual<second>", st);
    k_ozaki_residual<kWSX1, kWLmax><<<gres, 128, w_residual_smem(kWSX1, kWLmax), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R,
                                                                                      N, w.status);
  }
  {
    gw::TimedLaunch tl_("k_refine_update<double2>", st);
    k_refine_update<double2><<<gupd, 256, 0, st>>>(w.X1, w.R, mats, N);
  }
}

}  // namespace gw
