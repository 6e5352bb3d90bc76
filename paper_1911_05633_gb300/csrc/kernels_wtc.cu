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
#include "fpbits.h"
#include "ozaki.h"
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

// In-place FP32 Gauss-Jordan inverse with partial pivoting, one 512-thread block per
// matrix (N a multiple of kGJ32C, at most 512).  Panels of kGJ32B columns are reduced
// in shared memory, each warp owning every 16th row with one column per lane, two
// block barriers per column; the row exchanges and the rank-kGJ32B update of the other
// columns, A[:, T] += (Pan - I[:, panel]) Prow (Prow: the pivot rows before the
// update), run per chunk of kGJ32C columns with 8 x 4 complex register blocks per
// thread.  At the end the columns are permuted back by the composite of the pivot swaps.
__global__ void __launch_bounds__(512, 1)
k_gj_inverse_f32(float2* __restrict__ A, int N, long long mat_stride, int* __restrict__ status) {
  constexpr int B = kGJ32B, C = kGJ32C;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Pan = reinterpret_cast<float2*>(smraw);  // [N][B]
  float2* Buf = Pan + (size_t)N * B;               // Prow [B][C] / exchange staging [2B][C] / rows [16][N]
  int* pm = reinterpret_cast<int*>(Buf + gj32_buf_elems(N));  // [N] pivot row chosen for each column
  int* srcmap = pm + N;                            // [N]
  int* xdst = srcmap + N;                          // [2B]
  int* xsrc = xdst + 2 * B;                        // [2B]
  __shared__ float rv[2][16];  // pivot candidates per warp, by column parity
  __shared__ int ri[2][16];
  __shared__ int nx;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (N % C != 0 || N > 512) {
    if (tid == 0) atomicExch(status, 3);
    return;
  }
  float2* M = A + (long long)blockIdx.x * mat_stride;
  for (int k0 = 0; k0 < N; k0 += B) {
    for (int x = tid; x < N * B; x += 512) Pan[x] = M[(long long)(x / B) * N + k0 + (x % B)];
    __syncthreads();
    // pivot candidates of the panel's first column (at most one row per thread); those of
    // the later columns are gathered while the previous column is applied
    {
      float best = -1.0f;
      int bi = N;
      if (k0 + tid < N) {
        const float2 z = Pan[(k0 + tid) * B];
        best = fabsf(z.x) + fabsf(z.y);
        bi = k0 + tid;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { rv[0][wid] = best; ri[0][wid] = bi; }
    }
    __syncthreads();
    for (int m = 0; m < B; ++m) {
      const int k = k0 + m, par = m & 1;
      // every warp reduces the 16 candidates of column m itself (no barrier for the pivot)
      float best = lane < 16 ? rv[par][lane] : -1.0f;
      int bi = lane < 16 ? ri[par][lane] : N;
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const int p = bi < N ? bi : k;
      if (tid == 0) {
        pm[k] = p;
        if (!(best > 0.0f)) atomicExch(status, 1);
      }
      // lane j holds column j of the pivot row (scaled) and of the old row k
      const float2 d = Pan[p * B + m];
      const float den = d.x * d.x + d.y * d.y;
      const float2 inv = den > 0.0f ? make_float2(d.x / den, -d.y / den) : make_float2(0.0f, 0.0f);
      const float2 rowk = lane == m ? inv : cmul(Pan[p * B + lane], inv);
      const float2 oldk = Pan[k * B + lane];
      __syncthreads();  // rows p and k are read by every warp before their owners rewrite them
      // rows k and p exchanged and every row updated: warp w owns rows w, w + 16, ..., lane
      // = column; lane m + 1 keeps the pivot candidates of the next column below row k
      best = -1.0f;
      bi = N;
#pragma unroll 4
      for (int i = wid; i < N; i += 16) {
        const float2 cur = i == p ? oldk : Pan[i * B + lane];
        float2 v;
        if (i == k) {
          v = rowk;
        } else {
          const float2 f = make_float2(__shfl_sync(0xffffffffu, cur.x, m), __shfl_sync(0xffffffffu, cur.y, m));
          v = cfma(make_float2(-f.x, -f.y), rowk, lane == m ? make_float2(0.0f, 0.0f) : cur);
        }
        Pan[i * B + lane] = v;
        if (lane == m + 1 && i > k) {
          const float a = fabsf(v.x) + fabsf(v.y);
          if (a > best) { best = a; bi = i; }
        }
      }
      if (m + 1 < B && lane == m + 1) { rv[par ^ 1][wid] = best; ri[par ^ 1][wid] = bi; }
      __syncthreads();
    }
    // the trailing update below uses Pan - I on the panel's diagonal
    if (tid < B) Pan[(k0 + tid) * B + tid].x -= 1.0f;
    // composite row exchange of this panel: new row r = old row srcmap[r]
    for (int i = tid; i < N; i += 512) srcmap[i] = i;
    __syncthreads();
    if (wid == 0) {
      if (lane == 0)
        for (int m = 0; m < B; ++m) {
          const int k = k0 + m, p = pm[k];
          if (p != k) { const int t = srcmap[k]; srcmap[k] = srcmap[p]; srcmap[p] = t; }
        }
      __syncwarp();
      // the moved rows (at most 2B), compacted in row order
      int n = 0;
      for (int r0 = k0; r0 < N; r0 += 32) {
        const int r = r0 + lane;
        const bool mv = r < N && srcmap[r] != r;
        const unsigned bal = __ballot_sync(0xffffffffu, mv);
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        if (mv && pos < 2 * B) { xdst[pos] = r; xsrc[pos] = srcmap[r]; }
        n += __popc(bal);
      }
      if (lane == 0) nx = min(n, 2 * B);
    }
    __syncthreads();
    const int n = nx;
    for (int c0 = 0; c0 < N; c0 += C) {
      const bool has_panel = k0 >= c0 && k0 < c0 + C;
      // (a) the row exchange on this chunk's other columns, staged through shared memory
      for (int x = tid; x < n * C; x += 512) {
        const int e = x / C, j = c0 + (x % C);
        if (!(j >= k0 && j < k0 + B)) Buf[x] = M[(long long)xsrc[e] * N + j];
      }
      __syncthreads();
      for (int x = tid; x < n * C; x += 512) {
        const int e = x / C, j = c0 + (x % C);
        if (!(j >= k0 && j < k0 + B)) M[(long long)xdst[e] * N + j] = Buf[x];
      }
      __syncthreads();
      // (b) the pivot rows of this chunk before the update
      for (int x = tid; x < B * C; x += 512) Buf[x] = M[(long long)(k0 + x / C) * N + c0 + (x % C)];
      __syncthreads();
      // (c) rows i0 .. i0 + 7, columns c0 + lane + 32 q: 32 independent loads in flight per
      // thread, then 8 x 4 complex FMAs per pair of shared-memory vectors (z, pv)
      for (int i0 = 8 * wid; i0 < N; i0 += 8 * 16) {
        float2 acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = M[(long long)(i0 + r) * N + c0 + lane + 32 * q];
#pragma unroll 2
        for (int m = 0; m < B; ++m) {
          float2 z[8], pv[4];
#pragma unroll
          for (int r = 0; r < 8; ++r) z[r] = Pan[(i0 + r) * B + m];
#pragma unroll
          for (int q = 0; q < 4; ++q) pv[q] = Buf[m * C + lane + 32 * q];
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = cfma(z[r], pv[q], acc[r][q]);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = c0 + lane + 32 * q;
            if (!has_panel || !(j >= k0 && j < k0 + B)) M[(long long)(i0 + r) * N + j] = acc[r][q];
          }
      }
      __syncthreads();
    }
    if (tid < B) Pan[(k0 + tid) * B + tid].x += 1.0f;
    __syncthreads();
    for (int x = tid; x < N * B; x += 512) M[(long long)(x / B) * N + k0 + (x % B)] = Pan[x];
    __syncthreads();
  }
  // undo the pivoting on the columns: new column j = old column srcmap[j], the composite
  // of the swaps (k, pm[k]) for k = N-1 down to 0
  for (int i = tid; i < N; i += 512) srcmap[i] = i;
  __syncthreads();
  if (tid == 0)
    for (int k = N - 1; k >= 0; --k) {
      const int p = pm[k];
      if (p != k) { const int t = srcmap[k]; srcmap[k] = srcmap[p]; srcmap[p] = t; }
    }
  __syncthreads();
  float2* rb = Buf + (size_t)wid * N;
  for (int i = wid; i < N; i += 16) {
    float2* Mi = M + (long long)i * N;
    for (int j = lane; j < N; j += 32) rb[j] = Mi[j];
    __syncwarp();
    for (int j = lane; j < N; j += 32) Mi[j] = rb[srcmap[j]];
    __syncwarp();
  }
}

namespace {

using namespace umma;

constexpr uint64_t kWaitNs = 500ull * 1000ull * 1000ull;

}  // namespace

__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, long long n) {
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double2 z = src[x];
    dst[x] = make_float2((float)z.x, (float)z.y);
  }
}

// Scale exponents e with |x| < 2^e for every entry of a row of A (FP64) or of a column
// of X (FP32, or the unevaluated pair hi + lo), from the exponent fields alone: a normal
// x of biased exponent E has |x| < 2^(E - bias + 1).  0 for an all-zero row or column
// (subnormal entries count as zero).

// one warp per row
__global__ void k_row_exponent(const double2* __restrict__ A, int* __restrict__ eA, int N, int batch) {
  const int warps = blockDim.x >> 5;
  const long long row = (long long)blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= (long long)batch * N) return;
  const double2* a = A + row * N;
  int m = 0;
  for (int k = lane; k < N; k += 32) m = max(m, max(exp_field(a[k].x), exp_field(a[k].y)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) eA[row] = m > 0 ? m - 1022 : 0;
}

// one thread per column j (lo may be null): |hi|, |lo| < 2^(m - 126), so |hi + lo| < 2^(m - 125)
__global__ void k_col_exponent(const float2* __restrict__ hi, const float2* __restrict__ lo, int* __restrict__ eX,
                               int N) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const long long base = (long long)b * N * N + j;
  int m = 0;
  for (int k = 0; k < N; ++k) {
    const float2 h = hi[base + (long long)k * N];
    m = max(m, max(exp_field(h.x), exp_field(h.y)));
    if (lo) {
      const float2 l = lo[base + (long long)k * N];
      m = max(m, max(exp_field(l.x), exp_field(l.y)));
    }
  }
  eX[(long long)b * N + j] = m > 0 ? m - (lo ? 125 : 126) : 0;
}

// A operand digits.  Element (i, k) of matrix b -> kWSA digits of Re and of Im in the
// K-major tile layout, one chunk per (matrix, 128-row block, 16-wide K step) holding
// the 2 kWSA planes of 128 x 16 in the order (Re digits 0 .. kWSA-1, Im digits ...).
// One thread per (row i, 8 consecutive k): it reads 128 contiguous bytes and writes one
// 16-byte row of a core matrix per plane; the 32 lanes of a warp (i % 8, k half,
// (i / 8) % 2) fill 512 contiguous bytes of each plane.
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
      *reinterpret_cast<uint4*>(chunk + (0 * kWSA + s) * (128 * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (1 * kWSA + s) * (128 * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// X operand digits.  Element X[k][j] = hi + lo of matrix b (k = reduction index; lo may
// be null) -> SX digits of Re and of Im in the K-major layout of the B operand (rows j),
// one chunk per (matrix, kWTN-column block, 16-wide K step) holding the 2 SX planes of
// kWTN x 16 in the order (Re digits, Im digits).  One thread per (column j, 8
// consecutive k); lanes (j % 8, k half, (j / 8) % 2) read 128-byte row segments and fill
// 512 contiguous bytes of each plane.
template <int SX>
__global__ void k_slice_X(const float2* __restrict__ hi, const float2* __restrict__ lo, const int* __restrict__ eX,
                          uint16_t* __restrict__ Xsl, int N, long long n_total) {
  constexpr int JG = kWTN / 16;  // 16-column groups per block
  const int NKS = N / 16, NJB = N / kWTN;
  const long long n_thr = n_total / 8;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;  // (b, jb, ks, column group)
    const int jg = (int)(w % JG); w /= JG;
    const int ks = (int)(w % NKS); w /= NKS;
    const int jb = (int)(w % NJB);
    const long long b = w / NJB;
    const int h = (lane >> 3) & 1;
    const int jl = (lane & 7) + 8 * ((lane >> 4) + 2 * jg);  // column within the block
    const int j = jb * kWTN + jl;
    const int k0 = ks * 16 + 8 * h;
    const int e = eX[b * N + j];
    const long long o0 = (b * N + k0) * (long long)N + j;
    long long mr[8], mi[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 z = hi[o0 + (long long)u * N];
      mr[u] = fixed56(z.x, e);
      mi[u] = fixed56(z.y, e);
      if (lo) {  // each part rounds to 2^-56 of the column scale
        const float2 l = lo[o0 + (long long)u * N];
        mr[u] += fixed56(l.x, e);
        mi[u] += fixed56(l.y, e);
      }
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
      *reinterpret_cast<uint4*>(chunk + (0 * SX + t) * (kWTN * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (1 * SX + t) * (kWTN * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// Accumulator q (0..7) of one residual entry in units of 2^-52.  Accumulators 0..6
// hold exact multiples of 2^-14, 2^-21, 2^-28, 2^-35, 2^-35, 2^-42, 2^-42 below 2^24
// such units, so the scaled value is an exact integer (level 0 below 2^62); accumulator
// 7 (levels >= 5) is rounded to 2^-52.
__device__ __forceinline__ long long level_units52(float v, int q) {
  switch (q) {
    case 0: return (long long)__float2int_rn(v * 0x1p14f) << 38;
    case 1: return (long long)__float2int_rn(v * 0x1p21f) << 31;
    case 2: return (long long)__float2int_rn(v * 0x1p28f) << 24;
    case 3:
    case 4: return (long long)__float2int_rn(v * 0x1p35f) << 17;
    case 5:
    case 6: return (long long)__float2int_rn(v * 0x1p42f) << 10;
    default: return __float2ll_rn(v * 0x1p52f);
  }
}

// The residual as a real product of twice the length: the Re rows of A X are
// [Ar, -Ai] [Xr; Xi] and the Im rows [Ai, Ar] [Xr; Xi], so one output row (Re or Im)
// accumulates over 2N terms from one digit plane of A and one of X per 16-wide K step
// (-Ai through the negate-A bit of the instruction descriptor).  The products a_s x_t of
// level L = s + t go to accumulator q(L, half): levels 0, 1, 2 each one accumulator over
// both halves of K (<= 2 N terms), levels 3 and 4 one accumulator per half (<= N terms),
// levels >= 5 one accumulator.
__host__ __device__ constexpr int ozaki_bucket(int L, int half) {
  return L <= 2 ? L : L == 3 ? 3 + half : L == 4 ? 5 + half : 7;
}

// The MMAs of one 16-wide K step, fully unrolled.  `fresh` marks the accumulators whose
// first product of the whole K loop is in this step (written, not added).
template <int SX, int NA, int LMAX>
__device__ __forceinline__ void ozaki_issue_step(uint32_t tm, uint64_t da0, uint64_t dx0, uint32_t id, int half,
                                                 uint32_t fresh) {
  constexpr uint32_t PA = 128 * 16 * 2, PX = kWTN * 16 * 2;  // bytes per A / X plane
  uint32_t used = 0;
#pragma unroll
  for (int t = 0; t < SX; ++t) {
#pragma unroll
    for (int s = 0; s < NA; ++s) {
      if (s + t <= LMAX) {
        const int q = ozaki_bucket(s + t, half);
        const uint32_t acc = (((fresh & ~used) >> q) & 1u) ? 0u : 1u;
        used |= 1u << q;
        // descriptor start addresses are in 16-byte units in the low bits
        mma_bf16(tm + (uint32_t)q * kWTN, da0 + (uint64_t)((s * PA) >> 4), dx0 + (uint64_t)((t * PX) >> 4), id, acc);
      }
    }
  }
}

// R[b] = I - A[b] X[b] for one block of 128 output rows (Re rows for blockIdx.y < N/128,
// else Im rows) x kWTN columns per block (128 threads), from the A digits s <= LMAX and
// SX digits of X, products with s + t <= LMAX.  Eight FP32 accumulators of kWTN columns
// fill the 512 tensor-memory columns.  kWStages shared-memory stages; while step kk runs,
// the stage of step kk - 1 is refilled with step kk - 1 + kWStages.  The epilogue adds all
// levels and the identity as one exact 64-bit integer in units of 2^-52 (the levels
// cancel each other, so they are combined before any rounding), then rounds once to FP32
// (R is small; FP32 keeps it to 2^-24 of itself) into the Re or Im part of R.
template <int SX, int LMAX>
__global__ void __launch_bounds__(128, 1)
k_ozaki_residual(const uint16_t* __restrict__ Asl, const uint16_t* __restrict__ Xsl, const int* __restrict__ eA,
                 const int* __restrict__ eX, float2* __restrict__ R, int N, int* status) {
  static_assert(LMAX >= 5 && LMAX < kWSA, "every accumulator receives a product; A has kWSA digits");
  constexpr int NA = LMAX + 1;                            // A digits used
  constexpr uint32_t PA = 128 * 16 * 2, PX = kWTN * 16 * 2;
  constexpr uint32_t AB = NA * PA, XB = SX * PX, SB = AB + XB;  // bytes per stage
  constexpr uint32_t XC = wx_chunk(SX);
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[kWStages];
  __shared__ __align__(8) uint64_t mmad[kWStages];
  const int jb = blockIdx.x;
  const int NKS = N / 16, NIB = N / 128, NJB = N / kWTN;
  const bool imrow = (int)blockIdx.y >= NIB;
  const int ib = imrow ? (int)blockIdx.y - NIB : (int)blockIdx.y;
  const long long b = blockIdx.z;
  const int NK2 = 2 * NKS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kWStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&mmad[s], 1);
    }
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const unsigned char* Abase = reinterpret_cast<const unsigned char*>(Asl) + ((b * NIB + ib) * NKS) * (long long)kWAChunk;
  const unsigned char* Xbase = reinterpret_cast<const unsigned char*>(Xsl) + ((b * NJB + jb) * NKS) * (long long)XC;
  // step kk: half 0 takes (Ar | Ai for Im rows) with Xr, half 1 (Ai negated | Ar) with Xi
  auto load = [&](int kk, int st) {
    const int half = kk >= NKS ? 1 : 0, ks = kk - half * NKS;
    const int cA = imrow ? 1 - half : half;
    unsigned char* dst = sm + st * SB;
    mbar_arrive_expect_tx(&full[st], SB);
    bulk_g2s(dst, Abase + (long long)ks * kWAChunk + (long long)cA * kWSA * PA, AB, &full[st]);
    bulk_g2s(dst + AB, Xbase + (long long)ks * XC + (long long)half * SX * PX, XB, &full[st]);
  };
  bool ok = true;
  if (tid == 0) {
    const uint32_t id = idesc_bf16_f32(128, kWTN), idn = idesc_bf16_f32_negA(128, kWTN);
    const uint32_t s0 = smem_u32(sm);
    for (int s = 0; s < kWStages && s < NK2; ++s) load(s, s);
    for (int kk = 0; kk < NK2; ++kk) {
      const int st = kk % kWStages;
      if (!mbar_wait(&full[st], (uint32_t)(kk / kWStages) & 1u, kWaitNs, status)) { ok = false; break; }
      fence_after_sync();
      const int half = kk >= NKS ? 1 : 0;
      // first products: every accumulator at kk = 0, the second-half ones of levels 3, 4 at kk = NKS
      const uint32_t fresh = kk == 0 ? 0xFFu : (kk == NKS ? ((1u << 4) | (1u << 6)) : 0u);
      ozaki_issue_step<SX, NA, LMAX>(tm, smem_desc(s0 + st * SB, 128, 256), smem_desc(s0 + st * SB + AB, 128, 256),
                                     (!imrow && half) ? idn : id, half, fresh);
      mma_commit(&mmad[st]);
      if (kk >= 1 && kk - 1 + kWStages < NK2) {
        // the products of step kk - 1 are done once its commit arrives: refill its stage
        const int so = (kk - 1) % kWStages;
        if (!mbar_wait(&mmad[so], (uint32_t)((kk - 1) / kWStages) & 1u, kWaitNs, status)) { ok = false; break; }
        load(kk - 1 + kWStages, so);
      }
    }
  }
  // every thread waits for the last products; one outcome for the block
  const int last = NK2 - 1;
  const bool done = ok && mbar_wait(&mmad[last % kWStages], (uint32_t)(last / kWStages) & 1u, kWaitNs, status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 2);
  } else {
    const int i = ib * 128 + 32 * warp + lane;
    const int ea = eA[b * N + i];
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    // The pipeline stages are free now: each warp stages its 32 x 16 results there, so
    // that one store instruction covers two rows of 16 columns instead of 32 rows.
    float* stg = reinterpret_cast<float*>(sm) + warp * (32 * 17);
    float* Rw = reinterpret_cast<float*>(R + (b * N + ib * 128 + 32 * warp) * (long long)N) + (imrow ? 1 : 0);
    bool range_ok = true;
    for (int c0 = 0; c0 < kWTN; c0 += 16) {
      float v[128];  // accumulator q, column c at v[16 q + c]
      tmem_ld16x4(tm + lane_base + (uint32_t)c0, kWTN, v);
      tmem_ld16x4(tm + lane_base + (uint32_t)(4 * kWTN + c0), kWTN, v + 64);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        long long val = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) val += level_units52(v[16 * q + c], q);
        const int j = jb * kWTN + c0 + c;
        const int e = ea + eX[b * N + j];  // (A X)_ij = 2^e sum
        if (!imrow && i == j) {
          if (e < -10 || e > 52) range_ok = false;
          else val -= 1ll << (52 - e);  // 1 = 2^(52 - e) units of 2^(e - 52)
        }
        if (e < -126 || e > 126) range_ok = false;
        const float sc = __int_as_float((127 + min(max(e, -126), 126)) << 23);  // 2^e
        stg[lane * 17 + c] = -sc * ((float)val * 0x1p-52f);
      }
      __syncwarp();
#pragma unroll 4
      for (int t = 0; t < 16; ++t) {
        const int rr = 2 * t + (lane >> 4), cc = lane & 15;
        Rw[2 * ((long long)rr * N + jb * kWTN + c0 + cc)] = stg[rr * 17 + cc];
      }
      __syncwarp();
    }
    if (!range_ok) atomicExch(status, 4);  // scale outside the FP32 exponent range
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// Three BF16 terms of an FP32 value, v = hi + mid + lo to 2^-24 of |v| (each
// remainder is exact in FP32); bits of term s.
__device__ __forceinline__ void split3_bits(float v, uint32_t* t) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  const __nv_bfloat16 l = __float2bfloat16_rn(r2);
  t[0] = __bfloat16_as_ushort(h);
  t[1] = __bfloat16_as_ushort(m);
  t[2] = __bfloat16_as_ushort(l);
}

// 8 consecutive K elements of one operand row -> one 16-byte core-matrix row in each of
// the 6 planes (term s, Re/Im) of a kRefChunk chunk.
__device__ __forceinline__ void split3_store8(const float2* z, uint16_t* chunk, uint32_t off) {
  uint32_t tr[8][3], ti[8][3];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    split3_bits(z[u].x, tr[u]);
    split3_bits(z[u].y, ti[u]);
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    uint4 pr, pi;
    pr.x = tr[0][s] | (tr[1][s] << 16); pr.y = tr[2][s] | (tr[3][s] << 16);
    pr.z = tr[4][s] | (tr[5][s] << 16); pr.w = tr[6][s] | (tr[7][s] << 16);
    pi.x = ti[0][s] | (ti[1][s] << 16); pi.y = ti[2][s] | (ti[3][s] << 16);
    pi.z = ti[4][s] | (ti[5][s] << 16); pi.w = ti[6][s] | (ti[7][s] << 16);
    *reinterpret_cast<uint4*>(chunk + (s * 2 + 0) * (128 * 16) + off) = pr;
    *reinterpret_cast<uint4*>(chunk + (s * 2 + 1) * (128 * 16) + off) = pi;
  }
}

// BF16x3 operand planes of a row-major FP32 complex matrix M[b][r][k] (rows r = the MMA's
// M or N rows, k = reduction index): one kRefChunk chunk per (matrix, 128-row block,
// 16-wide K step).  Thread mapping as in k_slice_A.
__global__ void k_split3_rows(const float2* __restrict__ M, uint16_t* __restrict__ P, int N, long long n_total) {
  const int NKS = N / 16, NRB = N / 128;
  const long long n_thr = n_total / 8;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;
    const int gp = (int)(w % 8); w /= 8;
    const int ks = (int)(w % NKS); w /= NKS;
    const int rb = (int)(w % NRB);
    const long long b = w / NRB;
    const int h = (lane >> 3) & 1;
    const int rl = (lane & 7) + 8 * ((lane >> 4) + 2 * gp);
    const float2* src = M + (b * N + rb * 128 + rl) * (long long)N + ks * 16 + 8 * h;
    float2 z[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) z[u] = src[u];
    split3_store8(z, P + ((b * NRB + rb) * NKS + ks) * (long long)(kRefChunk / 2), kmajor_offset(128, rl, 8 * h) / 2);
  }
}

// The same planes for the transpose: element M[b][k][r] goes to row r (for the B operand
// of X R, whose rows are the columns of R).  Thread mapping as in k_slice_X.
__global__ void k_split3_cols(const float2* __restrict__ M, uint16_t* __restrict__ P, int N, long long n_total) {
  const int NKS = N / 16, NRB = N / 128;
  const long long n_thr = n_total / 8;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;
    const int gp = (int)(w % 8); w /= 8;
    const int ks = (int)(w % NKS); w /= NKS;
    const int rb = (int)(w % NRB);
    const long long b = w / NRB;
    const int h = (lane >> 3) & 1;
    const int rl = (lane & 7) + 8 * ((lane >> 4) + 2 * gp);
    const float2* src = M + (b * N + ks * 16 + 8 * h) * (long long)N + rb * 128 + rl;
    float2 z[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) z[u] = src[(long long)u * N];
    split3_store8(z, P + ((b * NRB + rb) * NKS + ks) * (long long)(kRefChunk / 2), kmajor_offset(128, rl, 8 * h) / 2);
  }
}

// D = X R for one 128 x 128 tile per block (128 threads) on tcgen05, from the BF16x3
// planes of X (A operand, rows i) and of R (B operand, rows j = columns of R): the six
// term products with s + t <= 2 for each of Re = Xr Rr - Xi Ri and Im = Xr Ri + Xi Rr,
// accumulated in FP32 in two 128-column tensor-memory accumulators.  R is small, so the
// product is needed to 2^-24 of itself only.  kRefStages shared-memory stages; while step
// ks runs, the stage of step ks - 1 is refilled with step ks - 1 + kRefStages.
//   MODE 0: lo[b] = D (X1 = X0 + lo is kept as the unevaluated FP32 pair)
//   MODE 1: out[b] = hi + lo + D in FP64
//   MODE 2: out[b] += D (a further refinement of the FP64 inverse in out)
template <int MODE>
__global__ void __launch_bounds__(128, 1)
k_refine_tc(const uint16_t* __restrict__ PX, const uint16_t* __restrict__ PR, const float2* __restrict__ hi,
            float2* __restrict__ lo, double2* __restrict__ out, int N, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[kRefStages];
  __shared__ __align__(8) uint64_t mmad[kRefStages];
  const int jb = blockIdx.x, ib = blockIdx.y;
  const long long b = blockIdx.z;
  const int NKS = N / 16, NRB = N / 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 256);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kRefStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&mmad[s], 1);
    }
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const unsigned char* Abase = reinterpret_cast<const unsigned char*>(PX) + ((b * NRB + ib) * NKS) * (long long)kRefChunk;
  const unsigned char* Bbase = reinterpret_cast<const unsigned char*>(PR) + ((b * NRB + jb) * NKS) * (long long)kRefChunk;
  constexpr uint32_t SB = 2 * kRefChunk;  // bytes per stage
  constexpr uint32_t PL = 128 * 16 * 2;   // bytes per plane
  bool ok = true;
  if (tid == 0) {
    const uint32_t id = idesc_bf16_f32(128, 128), idn = idesc_bf16_f32_negA(128, 128);
    const uint32_t s0 = smem_u32(sm);
    for (int s = 0; s < kRefStages && s < NKS; ++s) {
      mbar_arrive_expect_tx(&full[s], SB);
      bulk_g2s(sm + s * SB, Abase + (long long)s * kRefChunk, kRefChunk, &full[s]);
      bulk_g2s(sm + s * SB + kRefChunk, Bbase + (long long)s * kRefChunk, kRefChunk, &full[s]);
    }
    for (int ks = 0; ks < NKS; ++ks) {
      const int st = ks % kRefStages;
      if (!mbar_wait(&full[st], (uint32_t)(ks / kRefStages) & 1u, kWaitNs, status)) { ok = false; break; }
      fence_after_sync();
      const uint64_t da0 = smem_desc(s0 + st * SB, 128, 256), db0 = smem_desc(s0 + st * SB + kRefChunk, 128, 256);
      bool first = ks == 0;
#pragma unroll
      for (int sa = 0; sa < 3; ++sa) {
#pragma unroll
        for (int sb = 0; sb < 3; ++sb) {
          if (sa + sb <= 2) {
            const uint64_t dar = da0 + (uint64_t)(((sa * 2 + 0) * PL) >> 4), dai = da0 + (uint64_t)(((sa * 2 + 1) * PL) >> 4);
            const uint64_t dbr = db0 + (uint64_t)(((sb * 2 + 0) * PL) >> 4), dbi = db0 + (uint64_t)(((sb * 2 + 1) * PL) >> 4);
            const uint32_t acc = first ? 0u : 1u;
            mma_bf16(tm, dar, dbr, id, acc);          // Re += Xr Rr
            mma_bf16(tm, dai, dbi, idn, 1u);          // Re -= Xi Ri
            mma_bf16(tm + 128, dar, dbi, id, acc);    // Im += Xr Ri
            mma_bf16(tm + 128, dai, dbr, id, 1u);     // Im += Xi Rr
            first = false;
          }
        }
      }
      mma_commit(&mmad[st]);
      if (ks >= 1 && ks - 1 + kRefStages < NKS) {
        const int so = (ks - 1) % kRefStages;
        if (!mbar_wait(&mmad[so], (uint32_t)((ks - 1) / kRefStages) & 1u, kWaitNs, status)) { ok = false; break; }
        const int kn = ks - 1 + kRefStages;
        mbar_arrive_expect_tx(&full[so], SB);
        bulk_g2s(sm + so * SB, Abase + (long long)kn * kRefChunk, kRefChunk, &full[so]);
        bulk_g2s(sm + so * SB + kRefChunk, Bbase + (long long)kn * kRefChunk, kRefChunk, &full[so]);
      }
    }
  }
  const int last = NKS - 1;
  const bool done = ok && mbar_wait(&mmad[last % kRefStages], (uint32_t)(last / kRefStages) & 1u, kWaitNs, status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 2);
  } else {
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    // The pipeline stages are free now: each warp stages its 32 rows x 64 columns there,
    // so that its loads and stores run along rows (32 consecutive columns per instruction).
    float2* stg = reinterpret_cast<float2*>(sm) + warp * (32 * 65);
    const long long row0 = (b * N + ib * 128 + 32 * warp) * (long long)N + jb * 128;
    for (int c0 = 0; c0 < 128; c0 += 64) {
      float re[64], im[64];
      tmem_ld16x4(tm + lane_base + (uint32_t)c0, 16, re);
      tmem_ld16x4(tm + lane_base + (uint32_t)(128 + c0), 16, im);
#pragma unroll
      for (int c = 0; c < 64; ++c) stg[lane * 65 + c] = make_float2(re[c], im[c]);
      __syncwarp();
#pragma unroll 4
      for (int t = 0; t < 64; ++t) {
        const int rr = t >> 1, cc = 32 * (t & 1) + lane;
        const float2 z = stg[rr * 65 + cc];
        const long long o = row0 + (long long)rr * N + c0 + cc;
        if (MODE == 1) {
          const float2 h = hi[o], l = lo[o];
          out[o] = make_double2(f2d(h.x) + f2d(l.x) + f2d(z.x), f2d(h.y) + f2d(l.y) + f2d(z.y));
        } else if (MODE == 2) {
          const double2 x = out[o];
          out[o] = make_double2(x.x + f2d(z.x), x.y + f2d(z.y));
        } else {
          lo[o] = z;
        }
      }
      __syncwarp();
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

cudaError_t wtc_setup(size_t smem_gj32) {
  cudaError_t e = raise_smem_limit(k_gj_inverse_f32, smem_gj32);
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX0, kWL0>, w_residual_smem(kWSX0, kWL0));
  if (e == cudaSuccess) e = raise_smem_limit(k_ozaki_residual<kWSX1, kWLmax>, w_residual_smem(kWSX1, kWLmax));
  if (e == cudaSuccess) e = raise_smem_limit(k_refine_tc<0>, w_refine_smem());
  if (e == cudaSuccess) e = raise_smem_limit(k_refine_tc<1>, w_refine_smem());
  if (e == cudaSuccess) e = raise_smem_limit(k_refine_tc<2>, w_refine_smem());
  return e;
}

void wtc_inverse(const WtcBuffers& w, double2* mats, int batch, int N, size_t smem_gj32, cudaStream_t st,
                 int refinements) {
  const long long NN = (long long)N * N;
  const long long tot = (long long)batch * NN;
  const unsigned g1 = (unsigned)((tot + 255) / 256 < 65535LL * 8 ? (tot + 255) / 256 : 65535LL * 8);
  const long long t8 = tot / 8;  // slicing threads: one per 8 consecutive elements
  const unsigned g8 = (unsigned)((t8 + 255) / 256 < 65535LL * 8 ? (t8 + 255) / 256 : 65535LL * 8);
  const dim3 gcol((unsigned)((N + 127) / 128), (unsigned)batch);
  const dim3 gres((unsigned)(N / kWTN), (unsigned)(2 * (N / 128)), (unsigned)batch);  // Re rows, then Im rows
  const dim3 gref((unsigned)(N / 128), (unsigned)(N / 128), (unsigned)batch);
  // X0: FP32 Gauss-Jordan
  {
    gw::TimedLaunch tl_("k_to_f32", st);
    k_to_f32<<<g1, 256, 0, st>>>(mats, w.X32, tot);
  }
  {
    gw::TimedLaunch tl_("k_gj_inverse_f32", st);
    k_gj_inverse_f32<<<batch, 512, smem_gj32, st>>>(w.X32, N, NN, w.status);
  }
  // digits of A (kept for both residuals)
  {
    gw::TimedLaunch tl_("k_row_exponent", st);
    k_row_exponent<<<(unsigned)((batch * (long long)N + 7) / 8), 256, 0, st>>>(mats, w.eA, N, batch);
  }
  {
    gw::TimedLaunch tl_("k_slice_A", st);
    k_slice_A<<<g8, 256, 0, st>>>(mats, w.eA, w.Asl, N, tot);
  }
  // R0 = I - A X0 (FP32), lo = X0 R0: X1 = X0 + lo
  {
    gw::TimedLaunch tl_("k_col_exponent", st);
    k_col_exponent<<<gcol, 128, 0, st>>>(w.X32, nullptr, w.eX, N);
  }
  {
    gw::TimedLaunch tl_("k_slice_X", st);
    k_slice_X<kWSX0><<<g8, 256, 0, st>>>(w.X32, nullptr, w.eX, w.Xsl, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_ozaki_residual<first>", st);
    k_ozaki_residual<kWSX0, kWL0><<<gres, 128, w_residual_smem(kWSX0, kWL0), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R, N,
                                                                                  w.status);
  }
  {
    gw::TimedLaunch tl_("k_split3_rows", st);
    k_split3_rows<<<g8, 256, 0, st>>>(w.X32, w.PX, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_split3_cols", st);
    k_split3_cols<<<g8, 256, 0, st>>>(w.R, w.Xsl, N, tot);  // the X digits are no longer needed
  }
  {
    gw::TimedLaunch tl_("k_refine_tc<first>", st);
    k_refine_tc<0><<<gref, 128, w_refine_smem(), st>>>(w.PX, w.Xsl, w.X32, w.lo, nullptr, N, w.status);
  }
  // R1 = I - A X1 (FP32), X2 = X1 + X0 R1 in FP64, written over A
  {
    gw::TimedLaunch tl_("k_col_exponent", st);
    k_col_exponent<<<gcol, 128, 0, st>>>(w.X32, w.lo, w.eX, N);
  }
  {
    gw::TimedLaunch tl_("k_slice_X", st);
    k_slice_X<kWSX1><<<g8, 256, 0, st>>>(w.X32, w.lo, w.eX, w.Xsl, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_ozaki_residual<second>", st);
    k_ozaki_residual<kWSX1, kWLmax><<<gres, 128, w_residual_smem(kWSX1, kWLmax), st>>>(w.Asl, w.Xsl, w.eA, w.eX, w.R,
                                                                                      N, w.status);
  }
  {
    gw::TimedLaunch tl_("k_split3_cols", st);
    k_split3_cols<<<g8, 256, 0, st>>>(w.R, w.Xsl, N, tot);
  }
  {
    gw::TimedLaunch tl_("k_refine_tc<final>", st);
    k_refine_tc<1><<<gref, 128, w_refine_smem(), st>>>(w.PX, w.Xsl, w.X32, w.lo, mats, N, w.status);
  }
  // X <- X + X (I - A X) again, the left factor now the current X rounded to FP32 (the
  // correction is needed to 2^-24 of itself only): with X0 there the error would shrink
  // by |I - A X0| per step, with X by about kappa 2^-24 |I - A X|
  for (int r = 3; r <= refinements; ++r) {
    {
      gw::TimedLaunch tl_("k_to_f32", st);
      k_to_f32<<<g1, 256, 0, st>>>(mats, w.X32, tot);
    }
    {
      gw::TimedLaunch tl_("k_split3_rows", st);
      k_split3_rows<<<g8, 256, 0, st>>>(w.X32, w.PX, N, tot);
    }
    {
      gw::TimedLaunch tl_("k_panel_col_exp", st);
      k_panel_col_exp<<<dim3((unsigned)((N + 127) / 128), (unsigned)batch), 128, 0, st>>>(mats, NN, N, N, N, w.eX);
    }
    {
      gw::TimedLaunch tl_("k_slice_panel_B", st);
      k_slice_panel_B<<<g8, 256, 0, st>>>(mats, NN, N, w.eX, w.Xsl, N, N, t8);
    }
    {
      gw::TimedLaunch tl_("k_ozaki_residual<third>", st);
      k_ozaki_residual<kWSX1, kWLmax><<<gres, 128, w_residual_smem(kWSX1, kWLmax), st>>>(w.Asl, w.Xsl, w.eA, w.eX,
                                                                                        w.R, N, w.status);
    }
    {
      gw::TimedLaunch tl_("k_split3_cols", st);
      k_split3_cols<<<g8, 256, 0, st>>>(w.R, w.Xsl, N, tot);
    }
    {
      gw::TimedLaunch tl_("k_refine_tc<add>", st);
      k_refine_tc<2><<<gref, 128, w_refine_smem(), st>>>(w.PX, w.Xsl, w.X32, w.lo, mats, N, w.status);
    }
  }
}


// ---- Block Gauss-Jordan for N_PB beyond kWNmax --------------------------------------
//
// The inverse of an N x N matrix with N = nb bs (bs <= kWNmax) by Gauss-Jordan over
// blocks of bs rows and columns, without pivoting across blocks (the matrices of the W
// solve, v(q) and v(q)^-1 - P(q, i nu), are Hermitian positive definite, so every pivot
// block is too).  Pivot step k, with D = A_kk^-1 (the tensor-core inverse of bs x bs):
//   Rp = D A_k,:  (its block k replaced by I + D),
//   A_i,: -= A_ik Rp for every row block i != k   (so A_ik becomes -A_ik D),
//   A_k,: = Rp with block k = D.
// Every product has K = bs <= kWNmax terms, so it runs as the residual does: exact BF16
// digits of the two panels (per-row and per-column power-of-two scales), the level sums
// exact in FP32 tensor-memory accumulators, one exact 64-bit sum rounded once to FP64.

// Scale exponent of each row of an M x K panel (rows ld apart, matrices ms apart): one
// warp per row.
__global__ void k_panel_row_exp(const double2* __restrict__ A, long long ms, int ld, int M, int K, int batch,
                                int* __restrict__ e) {
  const int warps = blockDim.x >> 5;
  const long long row = (long long)blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= (long long)batch * M) return;
  const long long b = row / M, i = row % M;
  const double2* a = A + b * ms + i * ld;
  int m = 0;
  for (int k = lane; k < K; k += 32) m = max(m, max(exp_field(a[k].x), exp_field(a[k].y)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[row] = m > 0 ? m - 1022 : 0;
}

// Scale exponent of each column of a K x Nc panel: one thread per column.
__global__ void k_panel_col_exp(const double2* __restrict__ B, long long ms, int ld, int K, int Nc,
                                int* __restrict__ e) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nc) return;
  const double2* c = B + (long long)b * ms + j;
  int m = 0;
  for (int k = 0; k < K; ++k) {
    const double2 z = c[(long long)k * ld];
    m = max(m, max(exp_field(z.x), exp_field(z.y)));
  }
  e[(long long)b * Nc + j] = m > 0 ? m - 1022 : 0;
}

// A-operand digits of an M x K panel, chunks as k_slice_A: one per (matrix, 128-row
// block, 16-wide K step) with the kWSA digits of Re, then of Im.
__global__ void k_slice_panel_A(const double2* __restrict__ A, long long ms, int ld, const int* __restrict__ eA,
                                uint16_t* __restrict__ Asl, int M, int K, long long n_thr) {
  const int NKS = K / 16, NIB = M / 128;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;  // (b, ib, ks, row group pair)
    const int gp = (int)(w % 8); w /= 8;
    const int ks = (int)(w % NKS); w /= NKS;
    const int ib = (int)(w % NIB);
    const long long b = w / NIB;
    const int h = (lane >> 3) & 1;
    const int il = (lane & 7) + 8 * ((lane >> 4) + 2 * gp);
    const int i = ib * 128 + il;
    const int k0 = ks * 16 + 8 * h;
    const int e = eA[b * M + i];
    const double2* src = A + b * ms + (long long)i * ld + k0;
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
      *reinterpret_cast<uint4*>(chunk + (0 * kWSA + s) * (128 * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (1 * kWSA + s) * (128 * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// B-operand digits of a K x Nc panel (FP64), chunks as k_slice_X<kWSX1>: one per
// (matrix, kWTN-column block, 16-wide K step) with the kWSX1 digits of Re, then of Im.
__global__ void k_slice_panel_B(const double2* __restrict__ B, long long ms, int ld, const int* __restrict__ eB,
                                uint16_t* __restrict__ Bsl, int K, int Nc, long long n_thr) {
  constexpr int JG = kWTN / 16;
  const int NKS = K / 16, NJB = Nc / kWTN;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_thr; x += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(x & 31);
    long long w = x >> 5;  // (b, jb, ks, column group)
    const int jg = (int)(w % JG); w /= JG;
    const int ks = (int)(w % NKS); w /= NKS;
    const int jb = (int)(w % NJB);
    const long long b = w / NJB;
    const int h = (lane >> 3) & 1;
    const int jl = (lane & 7) + 8 * ((lane >> 4) + 2 * jg);
    const int j = jb * kWTN + jl;
    const int k0 = ks * 16 + 8 * h;
    const int e = eB[b * Nc + j];
    const double2* src = B + b * ms + (long long)k0 * ld + j;
    long long mr[8], mi[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 z = src[(long long)u * ld];
      mr[u] = fixed56(z.x, e);
      mi[u] = fixed56(z.y, e);
    }
    uint16_t* chunk = Bsl + ((b * NJB + jb) * NKS + ks) * (long long)(wx_chunk(kWSX1) / 2);
    const uint32_t off = kmajor_offset(kWTN, jl, 8 * h) / 2;
#pragma unroll
    for (int t = 0; t < kWSX1; ++t) {
      uint32_t pr[4], pi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t r0 = digit_bf16(next_digit(mr[2 * u], t), t), r1 = digit_bf16(next_digit(mr[2 * u + 1], t), t);
        const uint32_t i0 = digit_bf16(next_digit(mi[2 * u], t), t), i1 = digit_bf16(next_digit(mi[2 * u + 1], t), t);
        pr[u] = r0 | (r1 << 16);
        pi[u] = i0 | (i1 << 16);
      }
      *reinterpret_cast<uint4*>(chunk + (0 * kWSX1 + t) * (kWTN * 16) + off) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<uint4*>(chunk + (1 * kWSX1 + t) * (kWTN * 16) + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
    }
  }
}

// dst[b][r][c] = src[b][r][c] (+ 1 on the diagonal r == c when add_identity), r < rows,
// c < cols, for matrices of row strides sld / dld and matrix strides sms / dms.
__global__ void k_copy_panel(const double2* __restrict__ src, long long sms, int sld, double2* __restrict__ dst,
                             long long dms, int dld, int rows, int cols, int batch, int add_identity) {
  const long long per = (long long)rows * cols, n = per * batch;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const long long b = x / per, rc = x % per;
    const int r = (int)(rc / cols), c = (int)(rc % cols);
    double2 z = src[b * sms + (long long)r * sld + c];
    if (add_identity && r == c) z.x += 1.0;
    dst[b * dms + (long long)r * dld + c] = z;
  }
}


// Level L of a panel product (accumulator L) in units of 2^-52.  With K <= kWblkMaxK
// complex terms (2K real products per level) the sums of levels 0..5 are integers in their
// unit 2^-7(L+2) below 2^24, so exact in FP32; levels 6 and 7 are rounded there and here,
// far below 2^-52 of the scale.
__device__ __forceinline__ long long panel_units52(float v, int L) {
  switch (L) {
    case 0: return (long long)__float2int_rn(v * 0x1p14f) << 38;
    case 1: return (long long)__float2int_rn(v * 0x1p21f) << 31;
    case 2: return (long long)__float2int_rn(v * 0x1p28f) << 24;
    case 3: return (long long)__float2int_rn(v * 0x1p35f) << 17;
    case 4: return (long long)__float2int_rn(v * 0x1p42f) << 10;
    case 5: return (long long)__float2int_rn(v * 0x1p49f) << 3;
    default: return __float2ll_rn(v * 0x1p52f);
  }
}

// The MMAs of one 16-wide K step of a panel product: accumulator L holds level L, so for
// digit s of A the digits t = 0 .. 7 - s of B feed the consecutive accumulators s .. 7, and
// a run of up to four B planes (consecutive in shared memory) is one MMA of 64 x run
// columns: 11 MMAs per K step, each A plane read at most twice.
// `first`: the first K step, whose runs of digit 0 write their accumulators (every level
// has one) and the later runs add to them.
__device__ __forceinline__ void panel_issue_step(uint32_t tm, uint64_t da0, uint64_t dx0, bool neg, bool first) {
  constexpr uint32_t PA = 128 * 16 * 2, PX = kWTN * 16 * 2;  // bytes per A / B plane
#pragma unroll
  for (int s = 0; s <= kWLmax; ++s) {
#pragma unroll
    for (int t0 = 0; t0 <= kWLmax - s; t0 += 4) {
      const int n = (kWLmax - s - t0 + 1) < 4 ? (kWLmax - s - t0 + 1) : 4;
      const uint32_t id = neg ? idesc_bf16_f32_negA(128, kWTN * n) : idesc_bf16_f32(128, kWTN * n);
      mma_bf16(tm + (uint32_t)(s + t0) * kWTN, da0 + (uint64_t)((s * PA) >> 4), dx0 + (uint64_t)((t0 * PX) >> 4), id,
               (first && s == 0) ? 0u : 1u);
    }
  }
}

// C = A B (accumulate 0) or C = C - A B (accumulate 1) for an M x K panel A and a K x Nc
// panel B given as digits (k_slice_panel_A / _B), K <= kWblkMaxK, FP64 out.  Blocks of
// 128 output rows (Re rows for blockIdx.y < M/128, else Im rows) x kWTN columns, the
// products a_s b_t with s + t <= 7 in eight level accumulators (one per level, both K
// halves together); row blocks [skip0, skip1) are left alone.  The epilogue sums the
// levels as one exact 64-bit integer in units of 2^(eA + eB - 52), rounds it once to FP64
// and stages each warp's 32 x 16 results in shared memory so that a store covers two rows
// of 16 columns.
__global__ void __launch_bounds__(128, 1) k_oz_panel_gemm(const __grid_constant__ PanelGemmArgs g) {
  constexpr int SX = kWSX1, LMAX = kWLmax, NA = LMAX + 1;
  static_assert(LMAX == 7 && SX == 8, "eight levels, eight accumulators of kWTN columns");
  static_assert(NA <= kWSA, "A has kWSA digits");
  constexpr uint32_t PA = 128 * 16 * 2, PX = kWTN * 16 * 2;
  constexpr uint32_t AB = NA * PA, XB = SX * PX, SB = AB + XB;
  constexpr uint32_t XC = wx_chunk(SX);
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[kWStages];
  __shared__ __align__(8) uint64_t mmad[kWStages];
  const int jb = blockIdx.x;
  const int NKS = g.K / 16, NIB = g.M / 128, NJB = g.Nc / kWTN;
  const bool imrow = (int)blockIdx.y >= NIB;
  const int ib = imrow ? (int)blockIdx.y - NIB : (int)blockIdx.y;
  if (ib >= g.skip0 && ib < g.skip1) return;  // the whole block: before any barrier or allocation
  const long long b = blockIdx.z;
  const int NK2 = 2 * NKS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int* status = g.status;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kWStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&mmad[s], 1);
    }
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const unsigned char* Abase =
      reinterpret_cast<const unsigned char*>(g.Asl) + ((b * NIB + ib) * NKS) * (long long)kWAChunk;
  const unsigned char* Xbase = reinterpret_cast<const unsigned char*>(g.Bsl) + ((b * NJB + jb) * NKS) * (long long)XC;
  // step kk: half 0 takes (Ar | Ai for Im rows) with Br, half 1 (Ai negated | Ar) with Bi
  auto load = [&](int kk, int st) {
    const int half = kk >= NKS ? 1 : 0, ks = kk - half * NKS;
    const int cA = imrow ? 1 - half : half;
    unsigned char* dst = sm + st * SB;
    mbar_arrive_expect_tx(&full[st], SB);
    bulk_g2s(dst, Abase + (long long)ks * kWAChunk + (long long)cA * kWSA * PA, AB, &full[st]);
    bulk_g2s(dst + AB, Xbase + (long long)ks * XC + (long long)half * SX * PX, XB, &full[st]);
  };
  bool ok = true;
  if (tid == 0) {
    const uint32_t s0 = smem_u32(sm);
    for (int s = 0; s < kWStages && s < NK2; ++s) load(s, s);
    for (int kk = 0; kk < NK2; ++kk) {
      const int st = kk % kWStages;
      if (!mbar_wait(&full[st], (uint32_t)(kk / kWStages) & 1u, kWaitNs, status)) { ok = false; break; }
      fence_after_sync();
      const int half = kk >= NKS ? 1 : 0;
      panel_issue_step(tm, smem_desc(s0 + st * SB, 128, 256), smem_desc(s0 + st * SB + AB, 128, 256), !imrow && half,
                       kk == 0);
      mma_commit(&mmad[st]);
      if (kk >= 1 && kk - 1 + kWStages < NK2) {
        const int so = (kk - 1) % kWStages;
        if (!mbar_wait(&mmad[so], (uint32_t)((kk - 1) / kWStages) & 1u, kWaitNs, status)) { ok = false; break; }
        load(kk - 1 + kWStages, so);
      }
    }
  }
  const int last = NK2 - 1;
  const bool done = ok && mbar_wait(&mmad[last % kWStages], (uint32_t)(last / kWStages) & 1u, kWaitNs, status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 2);
  } else {
    const int i = ib * 128 + 32 * warp + lane;
    const int ea = g.eA[b * g.M + i];
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    double* stg = reinterpret_cast<double*>(sm) + warp * (32 * 17);
    double* Cw = reinterpret_cast<double*>(g.C + b * g.c_ms + (long long)(ib * 128 + 32 * warp) * g.ldc) + (imrow ? 1 : 0);
    const int* eBj = g.eB + b * g.Nc + jb * kWTN;
    for (int c0 = 0; c0 < kWTN; c0 += 16) {
      // this group's old C values and column exponents first: independent loads in flight
      // while the accumulators are read (a load after each store would wait out its latency)
      double cold[16];
      int eb[16];
      const int cc = lane & 15;
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int rr = 2 * t + (lane >> 4);
        cold[t] = g.accumulate ? Cw[2 * ((long long)rr * g.ldc + jb * kWTN + c0 + cc)] : 0.0;
        eb[t] = eBj[c0 + t];
      }
      float v[128];  // accumulator q, column c at v[16 q + c]
      tmem_ld16x4(tm + lane_base + (uint32_t)c0, kWTN, v);
      tmem_ld16x4(tm + lane_base + (uint32_t)(4 * kWTN + c0), kWTN, v + 64);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        long long val = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) val += panel_units52(v[16 * q + c], q);
        stg[lane * 17 + c] = i2d_scaled(val, ea + eb[c] - 52);
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int rr = 2 * t + (lane >> 4);
        const double pv = stg[rr * 17 + cc];
        Cw[2 * ((long long)rr * g.ldc + jb * kWTN + c0 + cc)] = g.accumulate ? cold[t] - pv : pv;
      }
      __syncwarp();
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}


namespace {

unsigned grid_for(long long n_thr) {
  const long long g = (n_thr + 255) / 256;
  return (unsigned)(g < 65535LL * 8 ? (g > 0 ? g : 1) : 65535LL * 8);
}

// C (M x Nc, rows ldc apart, matrices c_ms apart) = / -= A B for the panels A (M x K at
// A, rows lda apart) and B (K x Nc at B, rows ldb apart), every matrix of the batch.
void panel_gemm(const WblkBuffers& w, const double2* A, long long a_ms, int lda, const double2* B, long long b_ms,
                int ldb, double2* C, long long c_ms, int ldc, int M, int Nc, int K, int batch, int skip0, int skip1,
                int accumulate, cudaStream_t st) {
  {
    gw::TimedLaunch tl_("k_panel_row_exp", st);
    k_panel_row_exp<<<(unsigned)((batch * (long long)M + 7) / 8), 256, 0, st>>>(A, a_ms, lda, M, K, batch, w.eA);
  }
  {
    gw::TimedLaunch tl_("k_slice_panel_A", st);
    k_slice_panel_A<<<grid_for((long long)batch * M * K / 8), 256, 0, st>>>(A, a_ms, lda, w.eA, w.Asl, M, K,
                                                                             (long long)batch * M * K / 8);
  }
  {
    gw::TimedLaunch tl_("k_panel_col_exp", st);
    k_panel_col_exp<<<dim3((unsigned)((Nc + 127) / 128), (unsigned)batch), 128, 0, st>>>(B, b_ms, ldb, K, Nc, w.eB);
  }
  {
    gw::TimedLaunch tl_("k_slice_panel_B", st);
    k_slice_panel_B<<<grid_for((long long)batch * K * Nc / 8), 256, 0, st>>>(B, b_ms, ldb, w.eB, w.Bsl, K, Nc,
                                                                              (long long)batch * K * Nc / 8);
  }
  PanelGemmArgs g{};
  g.Asl = w.Asl;
  g.Bsl = w.Bsl;
  g.eA = w.eA;
  g.eB = w.eB;
  g.C = C;
  g.c_ms = c_ms;
  g.ldc = ldc;
  g.M = M;
  g.Nc = Nc;
  g.K = K;
  g.skip0 = skip0;
  g.skip1 = skip1;
  g.accumulate = accumulate;
  g.status = w.inner.status;
  {
    gw::TimedLaunch tl_("k_oz_panel_gemm", st);
    k_oz_panel_gemm<<<dim3((unsigned)(Nc / kWTN), (unsigned)(2 * (M / 128)), (unsigned)batch), 128,
                      w_residual_smem(kWSX1, kWLmax), st>>>(g);
  }
}

void copy_panel(const double2* src, long long sms, int sld, double2* dst, long long dms, int dld, int rows, int cols,
                int batch, int add_identity, cudaStream_t st) {
  gw::TimedLaunch tl_("k_copy_panel", st);
  k_copy_panel<<<grid_for((long long)batch * rows * cols), 256, 0, st>>>(src, sms, sld, dst, dms, dld, rows, cols,
                                                                          batch, add_identity);
}

}  // namespace

int wblk_block_size(int N) {
  if (N <= kWNmax || N % 128 != 0) return 0;
  for (int bs = kWblkMaxK; bs >= 128; bs -= 128)
    if (N % bs == 0) return bs;
  return 0;
}

cudaError_t wblk_setup(size_t smem_gj32_bs) {
  cudaError_t e = wtc_setup(smem_gj32_bs);
  if (e == cudaSuccess) e = raise_smem_limit(k_oz_panel_gemm, w_residual_smem(kWSX1, kWLmax));
  return e;
}

void wblk_inverse(const WblkBuffers& w, double2* mats, int batch, int N, int bs, size_t smem_gj32_bs,
                  cudaStream_t st) {
  const long long NN = (long long)N * N, BB = (long long)bs * bs, BN = (long long)bs * N;
  for (int k = 0; k < N / bs; ++k) {
    const int r0 = k * bs;
    // D = A_kk^-1
    copy_panel(mats + (long long)r0 * N + r0, NN, N, w.D, BB, bs, bs, bs, batch, 0, st);
    wtc_inverse(w.inner, w.D, batch, bs, smem_gj32_bs, st, kWblkRefinements);
    // Rp = D A_k,: with block k = I + D
    panel_gemm(w, w.D, BB, bs, mats + (long long)r0 * N, NN, N, w.Rp, BN, N, bs, N, bs, batch, 0, 0, 0, st);
    copy_panel(w.D, BB, bs, w.Rp + r0, BN, N, bs, bs, batch, 1, st);
    // A_i,: -= A_ik Rp for the other row blocks (the column panel is sliced before any write)
    panel_gemm(w, mats + r0, NN, N, w.Rp, BN, N, mats, NN, N, N, N, bs, batch, r0 / 128, (r0 + bs) / 128, 1, st);
    // A_k,: = Rp with block k = D
    copy_panel(w.Rp, BN, N, mats + (long long)r0 * N, NN, N, bs, N, batch, 0, st);
    copy_panel(w.D, BB, bs, mats + (long long)r0 * N + r0, NN, N, bs, bs, batch, 0, st);
  }
}

}  // namespace gw
