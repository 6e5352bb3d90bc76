// Structured bosonic tau <-> i nu transforms of the product-basis layout (App. A grid,
// Sec. 2 layout) as one fused, persistent tensor-core kernel per transform:
//
//   P(R, i nu_m)  = sum_i a_mi Re P(R, tau_i) + b_mi Im P(R, tau_i)     (mirror-paired input)
//   W~(R, tau_i)  = sum_m T^-1_im W~(R, i nu_m)                          (real input)
//
// Rows are the K_a K_b elements of every pair entry, 128 per tile; the reduction runs over
// the input slices, the columns over the outputs.  Each CTA (one per SM) streams its tiles
// straight from HBM:
//   * eight slicer warps load a tile's FP64 values, take each row's power-of-two scale and
//     cut the scaled values into eight balanced base-2^7 digits, which BF16 holds exactly,
//     and write them to a ring of shared-memory stages (one 16-wide K step per stage);
//   * one thread issues the digit products on tcgen05 against the column operand's digits,
//     which stay resident in shared memory for the whole kernel;
//   * eight epilogue warps read the per-level FP32 accumulators from tensor memory, add the
//     levels as one exact 64-bit integer and round once to FP64.
// The digit products of level L = s + t (digit s of a row, digit t of a column) go to one
// accumulator per level; consecutive digit planes of the column operand sit next to each
// other in shared memory, so one MMA of width (planes x NT) feeds consecutive levels.  With
// a reduction of at most 80 terms every level's partial sums are integers (in its unit)
// below 2^22, exact whatever rounding the tensor core applies; when 8 levels do not fit
// the 512 tensor-memory columns, levels >= 5 share the last accumulator (rounded there, at
// 2^-50 of the scale).  The result has the error of an FP64 dot product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "ktimer.h"
#include "oz.h"
#include "ozaki.h"
#include "smem_limit.h"
#include "umma.h"

namespace gw {

namespace {

using namespace umma;

constexpr uint64_t kTfWaitNs = 500ull * 1000ull * 1000ull;
constexpr int kTfSlicerWarps = 8;                                    // 16 rows x 2 K halves each
constexpr int kTfEpiWarps = 8;                                       // 2 per tensor-memory lane quadrant
constexpr int kTfMmaWarp = kTfSlicerWarps;                           // warp 8
constexpr int kTfThreads = 32 * (kTfSlicerWarps + 1 + kTfEpiWarps);  // 544
constexpr int kTfSlicers = 32 * kTfSlicerWarps;
constexpr int kTfEpis = 32 * kTfEpiWarps;
constexpr uint32_t kTfPlane = 128 * 16 * 2;        // one digit plane of a 128 x 16 K step
constexpr uint32_t kTfAStage = kOzDigits * kTfPlane;  // 32 KB
constexpr int kTfMaxKS = 5;                        // reduction <= 80 terms with the values held
constexpr int kTfMaxKSGeneral = 8;                 // reduction <= 128 terms (values loaded again)
constexpr int kTfMaxNT = 80;                       // columns <= 80
// 64 in every base-2^7 position below the top one: m + kTfBias has non-negative 7-bit
// fields u_s, and m = t_0 2^49 + sum_{s>=1} (u_s - 64) 2^(49 - 7 s) with balanced digits.
constexpr long long kTfBias = 64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) +
                                      (1ll << 7) + 1ll);

// Tensor-memory accumulators: one per level up to nslot - 1, the last one takes the rest.
__host__ __device__ constexpr int tf_nslot(int NT) { return 512 / NT >= 8 ? 8 : 512 / NT; }

struct TfArgs {
  const DevEntry* ent;
  const int* tile_e;   // [n_rt] entry of a 128-row tile
  const int* tile_r0;  // [n_rt] its first element within the entry's block
  int n_rt;            // row tiles; the work is n_rt x n_ct tiles, column tile major
  int n_ct;            // column tiles of NT columns
  int pb;              // 1: product-basis blocks (K_a K_b), 0: orbital blocks (n_a n_b)
  const double2* in;   // input, n_in slices per entry block
  int n_in;
  int K;               // reduction length (values per row)
  int real_in;         // 1: value k = Re in[k]; 0: value 2i + c = component c of in[i]
  double2* out;        // output, n_out slices per entry block
  int n_out;
  int out_slice0;      // column n (kTfOutReal) goes to output slice out_slice0 + n
  int out_mode;        // kTfOut*
  int n_cols;          // columns of the column operand (all column tiles)
  int NT;              // columns per tile and accumulator (multiple of 16)
  const uint16_t* Bdig;  // per column tile [KS][kOzDigits][NT x 16] in the K-major layout
  const int* eB;         // [n_ct NT] column scale exponents
  int* status;
};

// Where the columns go: the real part of output slice n (imaginary part 0); or columns
// 2m + c as component c of output slice m; or that and slice n_out - 1 - m as its conjugate.
constexpr int kTfOutReal = 0;
constexpr int kTfOutComplex = 1;
constexpr int kTfOutMirror = 2;
constexpr int kTfMaxCols = 160;  // columns of all column tiles

// BF16 bits (upper half of the FP32 word) of balanced digit s of a scaled value, from
// M = m + kTfBias: s = 0 gives t_0 = floor(M / 2^49) (|t_0| <= 128), s >= 1 gives
// (u_s - 64) 2^-7s with u_s the 7-bit field of M at bit 49 - 7 s.  Every digit has at most
// 8 significant bits, so its FP32 form has a zero low half and the top half is exact BF16.
template <int s>
__device__ __forceinline__ uint32_t tf_digit(long long M) {
  if (s == 0) return __float_as_uint(__int_as_float(0x4B400000 + (int)(M >> 49)) - 12582912.0f);  // 1.5 2^23 + t0
  const uint32_t u = (uint32_t)((unsigned long long)M >> (49 - 7 * s)) & 127u;
  const float sc = __int_as_float((127 - 7 * s) << 23);  // 2^-7s
  // (2^23 + u) 2^-7s - (2^23 + 64) 2^-7s = (u - 64) 2^-7s, exact in one FMA
  return __float_as_uint(fmaf(__int_as_float(0x4B000000 | u), sc, -8388672.0f * sc));
}

// The 16-byte core-matrix row of digit plane s for 8 consecutive values.
template <int s>
__device__ __forceinline__ uint4 tf_plane_row(const long long* M) {
  return make_uint4(__byte_perm(tf_digit<s>(M[0]), tf_digit<s>(M[1]), 0x7632),
                    __byte_perm(tf_digit<s>(M[2]), tf_digit<s>(M[3]), 0x7632),
                    __byte_perm(tf_digit<s>(M[4]), tf_digit<s>(M[5]), 0x7632),
                    __byte_perm(tf_digit<s>(M[6]), tf_digit<s>(M[7]), 0x7632));
}

// Adds accumulator l to the 64-bit sums S (units of 2^-52 of the scale).  Accumulator l
// holds sum d_s d_t 2^-7L over its level(s); the digits carry 2^7 each, so the value in
// units of 2^-52 is v 2^38.  A single level's v 2^7L is an integer below 2^22, read exactly
// by adding 1.5 2^23 (one FMA and one integer subtraction: no float-to-integer conversion,
// which this chip runs at its FP64 rate).  The shared last accumulator (levels >= 5, below
// 2^25 in units of 2^-52) is split at a multiple of 8 and both parts read the same way.
__device__ __forceinline__ void tf_add_level(long long* S, const float* v, int l, bool shared) {
  if (!shared) {
    const float sc = __int_as_float((127 + 7 * l) << 23);  // 2^7l
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int I = __float_as_int(fmaf(v[j], sc, 12582912.0f)) - 0x4B400000;
      if (l <= 5) S[j] += (long long)I << (38 - 7 * l);
      else S[j] += (long long)((I + (1 << (7 * l - 39))) >> (7 * l - 38));  // rounded, half up
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float x = v[j] * 0x1p38f;                    // |x| < 2^25
      const float y = x + 100663296.0f;                  // 1.5 2^26: x rounded to a multiple of 8
      const int hi = __float_as_int(y) - 0x4CC00000;     // that multiple / 8
      const float lo = x - (y - 100663296.0f);           // exact, |lo| <= 4
      const int il = __float_as_int(lo + 12582912.0f) - 0x4B400000;
      S[j] += ((long long)hi << 3) + il;
    }
  }
}

// Reads accumulator l into the 64-bit sums as tf_add_level, for level sums that may reach
// 2^24 (reductions beyond 102 terms): the integer is split at a multiple of 4 first.
__device__ __forceinline__ void tf_add_level_wide(long long* S, const float* v, int l) {
  const float sc = __int_as_float((127 + 7 * l) << 23);  // 2^7l
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float x = v[j] * sc;                          // an integer, |x| < 2^24
    const float y = x + 50331648.0f;                    // 1.5 2^25 (y in one binade): x to a multiple of 4
    const int hi = __float_as_int(y) - 0x4C400000;      // that multiple / 4
    const int I = 4 * hi + (__float_as_int((x - (y - 50331648.0f)) + 12582912.0f) - 0x4B400000);
    if (l <= 5) S[j] += (long long)I << (38 - 7 * l);
    else S[j] += (long long)((I + (1 << (7 * l - 39))) >> (7 * l - 38));
  }
}

// The digit products of one K step for columns NT wide, as a schedule fixed at compile
// time: digit s of the rows against digits t .. t + cnt - 1 of the columns (consecutive
// planes, one MMA cnt NT wide) into accumulators slot .. slot + cnt - 1; `init`: the MMA
// writes (does not add to) its accumulators in the first K step of a tile.
struct TfMma {
  int s, t, cnt, slot, init;
};
template <int NT>
struct TfSchedule {
  TfMma m[kOzDigits * kOzDigits];
  int n;
  constexpr TfSchedule() : m(), n(0) {
    const int nslot = tf_nslot(NT);
    unsigned inited = 0;
    for (int s = 0; s < kOzDigits; ++s)
      for (int t = 0; t <= kOzLmax - s;) {
        const int slot = s + t < nslot - 1 ? s + t : nslot - 1;
        int cnt = 1;
        while (t + cnt <= kOzLmax - s && (s + t + cnt < nslot - 1 ? s + t + cnt : nslot - 1) == slot + cnt &&
               (cnt + 1) * NT <= 256)
          ++cnt;
        m[n].s = s;
        m[n].t = t;
        m[n].cnt = cnt;
        m[n].slot = slot;
        m[n].init = ((inited >> slot) & 1u) ? 0 : 1;
        inited |= ((1u << cnt) - 1u) << slot;
        ++n;
        t += cnt;
      }
  }
};

// Issues the digit products of one K step: dA, dB the descriptors of the step's first row
// and column digit planes (planes kTfPlane and NT x 32 bytes apart: the descriptor's address
// field counts 16-byte units).
template <int NT>
__device__ __forceinline__ void tf_issue_step(uint32_t tm, uint64_t dA, uint64_t dB, bool first) {
  constexpr TfSchedule<NT> S{};
#pragma unroll
  for (int i = 0; i < S.n; ++i) {
    const TfMma m = S.m[i];
    mma_bf16(tm + (uint32_t)(m.slot * NT), dA + (uint64_t)(m.s * (kTfPlane >> 4)),
             dB + (uint64_t)(m.t * (NT * 32 / 16)), idesc_bf16_f32(128, m.cnt * NT), (first && m.init) ? 0u : 1u);
  }
}
__device__ __forceinline__ void tf_issue(int NT, uint32_t tm, uint64_t dA, uint64_t dB, bool first) {
  switch (NT) {
    case 16: tf_issue_step<16>(tm, dA, dB, first); break;
    case 32: tf_issue_step<32>(tm, dA, dB, first); break;
    case 48: tf_issue_step<48>(tm, dA, dB, first); break;
    case 64: tf_issue_step<64>(tm, dA, dB, first); break;
    default: tf_issue_step<80>(tm, dA, dB, first); break;
  }
}

// Exact integer of a single level's accumulator value v 2^7l (|.| <= 2^22, or < 2^24 WIDE).
template <bool WIDE>
__device__ __forceinline__ int tf_level_int(float v, float sc) {
  if (!WIDE) return __float_as_int(fmaf(v, sc, 12582912.0f)) - 0x4B400000;
  const float x = v * sc;
  const float y = x + 50331648.0f;
  return 4 * (__float_as_int(y) - 0x4C400000) + (__float_as_int((x - (y - 50331648.0f)) + 12582912.0f) - 0x4B400000);
}

// Adds the single levels l and l + 1 (two accumulators read together) to the 64-bit sums:
// I_l 2^7 + I_{l+1} is a 32-bit integer, shifted once into units of 2^-52 (levels 6 and 7:
// rounded, half up, at 2^-52).
template <bool WIDE>
__device__ __forceinline__ void tf_add_pair(long long* S, const float* v, int l) {
  const float s0 = __int_as_float((127 + 7 * l) << 23), s1 = __int_as_float((127 + 7 * (l + 1)) << 23);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int P = tf_level_int<WIDE>(v[j], s0) * 128 + tf_level_int<WIDE>(v[16 + j], s1);
    if (l + 1 <= 5) S[j] += (long long)P << (38 - 7 * (l + 1));
    else S[j] += (long long)((P + 1024) >> 11);  // l = 6: I_6 2^-4 + I_7 2^-11
  }
}

// WIDE: level sums may exceed 2^22 (reductions beyond 102 terms).
// STAGE: the epilogue stages its 64-bit sums in shared memory and releases the tensor
// memory before converting and storing them (two A stages instead of three).
template <int KS, bool WIDE, bool STAGE>
__global__ void __launch_bounds__(kTfThreads, 1) k_oz_transform(const __grid_constant__ TfArgs g) {
  constexpr int kTfStages = STAGE ? 2 : 3;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t a_full[kTfStages], a_empty[kTfStages];
  __shared__ __align__(8) uint64_t t_full, t_empty, b_full, b_free, drained;
  __shared__ __align__(8) uint64_t e_full[2], e_empty[2];
  __shared__ int eA_s[2][128];
  __shared__ int eB_s[kTfMaxCols];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NT = g.NT, nslot = tf_nslot(NT);
  const uint32_t BK = (uint32_t)kOzDigits * NT * 32;  // column digits of one K step
  unsigned char* Bs = sm;
  unsigned char* As = sm + KS * BK;
  long long* Ss = reinterpret_cast<long long*>(As + kTfStages * kTfAStage);  // STAGE: [NT][128]
  if (warp == kTfMmaWarp) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTfStages; ++s) {
      mbar_init(&a_full[s], kTfSlicers);
      mbar_init(&a_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&e_full[b], kTfSlicers);
      mbar_init(&e_empty[b], kTfEpis);
    }
    mbar_init(&t_full, 1);
    mbar_init(&t_empty, kTfEpis);
    mbar_init(&b_full, 1);
    mbar_init(&b_free, 1);
    mbar_init(&drained, 1);
    fence_mbar_init();
  }
  for (int n = threadIdx.x; n < g.n_ct * NT; n += blockDim.x) eB_s[n] = g.eB[n];
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const int n_tiles = g.n_rt * g.n_ct;
  const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto entry_of = [&](int t, DevEntry& E, long long& blk, long long& base, int& r0, int& ct) {
    ct = t / g.n_rt;
    const int rt = t - ct * g.n_rt;
    E = g.ent[g.tile_e[rt]];
    blk = g.pb ? (long long)E.Ka * E.Kb : (long long)E.na * E.nb;
    base = g.pb ? E.off_pb : E.off_orb;
    r0 = g.tile_r0[rt];
  };

  if (warp < kTfSlicerWarps) {
    // ---- slicers: row r of the tile, K half h of every 16-wide step ----
    const int r = 16 * warp + (lane & 15), h = lane >> 4;
    int step = 0;
    bool ok = true;
    for (int i = 0; i < my_tiles && ok; ++i) {
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      DevEntry E;
      long long blk, base;
      int r0, ct;
      entry_of(t, E, blk, base, r0, ct);
      const long long x = r0 + r;
      const bool valid = x < blk;
      if (warp == 0 && lane == 0 && i + 1 < my_tiles) {
        // the next tile's input, into L2 while this one is cut
        DevEntry En;
        long long bn, basen;
        int rn, ctn;
        entry_of(t + (int)gridDim.x, En, bn, basen, rn, ctn);
        const uint32_t bytes = (uint32_t)(min(128ll, bn - rn) * 16);
        const int ns = g.real_in ? g.K : (g.K + 1) / 2;
        for (int k = 0; k < ns; ++k) prefetch_l2(g.in + basen * g.n_in + k * bn + rn, bytes);
      }
      const double2* src = g.in + base * g.n_in + x;
      // the 8 values of this thread in K step ks
      auto load8 = [&](int ks, double* w) {
        if (g.real_in) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = ks * 16 + 8 * h + u;
            w[u] = (valid && k < g.K) ? reinterpret_cast<const double*>(src + k * blk)[0] : 0.0;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int sl = ks * 8 + 4 * h + j;  // values 2 sl, 2 sl + 1
            double2 p = make_double2(0.0, 0.0);
            if (valid && 2 * sl < g.K) p = src[sl * blk];
            w[2 * j] = p.x;
            w[2 * j + 1] = p.y;
          }
        }
      };
      // one K step cut into its stage: the digit planes of 8 values of this thread
      auto cut = [&](const double* w, int e, int st) {
        unsigned char* A = As + st * kTfAStage + kmajor_offset(128, r, 8 * h);
        long long M[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) M[u] = fixed56(w[u], e) + kTfBias;
        *reinterpret_cast<uint4*>(A + 0 * kTfPlane) = tf_plane_row<0>(M);
        *reinterpret_cast<uint4*>(A + 1 * kTfPlane) = tf_plane_row<1>(M);
        *reinterpret_cast<uint4*>(A + 2 * kTfPlane) = tf_plane_row<2>(M);
        *reinterpret_cast<uint4*>(A + 3 * kTfPlane) = tf_plane_row<3>(M);
        *reinterpret_cast<uint4*>(A + 4 * kTfPlane) = tf_plane_row<4>(M);
        *reinterpret_cast<uint4*>(A + 5 * kTfPlane) = tf_plane_row<5>(M);
        *reinterpret_cast<uint4*>(A + 6 * kTfPlane) = tf_plane_row<6>(M);
        *reinterpret_cast<uint4*>(A + 7 * kTfPlane) = tf_plane_row<7>(M);
        fence_smem_to_async();
        mbar_arrive(&a_full[st]);
      };
      // the scale pass, one K step at a time; the cut reads the values again (from L2)
      int mx = 0;
#pragma unroll 1
      for (int ks = 0; ks < KS; ++ks) {
        double w[8];
        load8(ks, w);
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = max(mx, exp_field(w[u]));
      }
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
      const int e = mx > 0 ? mx - 1022 : 0;
      const int b = i & 1;
      ok = mbar_wait(&e_empty[b], (uint32_t)((i >> 1) & 1) ^ 1u, kTfWaitNs, g.status);
      if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
      if (h == 0) eA_s[b][r] = e;
      mbar_arrive(&e_full[b]);
#pragma unroll 1
      for (int ks = 0; ks < KS; ++ks, ++step) {
        double w[8];
        load8(ks, w);
        const int st = step % kTfStages;
        ok = mbar_wait(&a_empty[st], (uint32_t)((step / kTfStages) & 1) ^ 1u, kTfWaitNs, g.status);
        if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
        cut(w, e, st);
      }
    }
    if (!ok) atomicExch(g.status, 2);
  } else if (warp == kTfMmaWarp) {
    // ---- one thread issues the digit products ----
    if (lane == 0) {
      bool ok = true;
      const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
      int step = 0, cur_ct = -1, b_loads = 0;
      for (int i = 0; i < my_tiles && ok; ++i) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        const int ct = t / g.n_rt;
        if (ct != cur_ct) {
          // a new column tile: its digits replace the resident ones once every product
          // issued so far has read them
          if (b_loads > 0) {
            mma_commit(&b_free);
            if (!(ok = mbar_wait(&b_free, (uint32_t)((b_loads - 1) & 1), kTfWaitNs, g.status))) break;
          }
          mbar_arrive_expect_tx(&b_full, KS * BK);
          const unsigned char* src = reinterpret_cast<const unsigned char*>(g.Bdig) + (size_t)ct * KS * BK;
          for (int ks = 0; ks < KS; ++ks) bulk_g2s(Bs + ks * BK, src + (size_t)ks * BK, BK, &b_full);
          if (!(ok = mbar_wait(&b_full, (uint32_t)(b_loads & 1), kTfWaitNs, g.status))) break;
          ++b_loads;
          cur_ct = ct;
        }
        if (!(ok = mbar_wait(&t_empty, (uint32_t)(i & 1) ^ 1u, kTfWaitNs, g.status))) break;
        fence_after_sync();
        for (int ks = 0; ks < KS && ok; ++ks, ++step) {
          const int st = step % kTfStages;
          ok = mbar_wait(&a_full[st], (uint32_t)((step / kTfStages) & 1), kTfWaitNs, g.status);
          if (!ok) break;
          fence_after_sync();
          tf_issue(NT, tm, smem_desc(a_base + st * kTfAStage, 128, 256), smem_desc(b_base + ks * BK, 128, 256),
                   ks == 0);
          mma_commit(&a_empty[st]);
        }
        if (ok) mma_commit(&t_full);
      }
      // every product issued has finished before the accumulators are released
      mma_commit(&drained);
      if (!mbar_wait(&drained, 0, kTfWaitNs, nullptr)) ok = false;
      if (!ok) atomicExch(g.status, 2);
    }
  } else {
    // ---- epilogue: TMEM lane quadrant q, 16-column chunks c = half, half + 2, ... ----
    const int q = warp & 3, half = (warp - kTfMmaWarp - 1) >> 2;
    const int row = 32 * q + lane;
    const int n_chunks = NT / 16;
    const int last_c = ((n_chunks - 1 - half) / 2) * 2 + half;  // this warp's last chunk
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int i = 0; i < my_tiles && ok; ++i) {
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      DevEntry E;
      long long blk, base;
      int r0, ct;
      entry_of(t, E, blk, base, r0, ct);
      const long long x = r0 + row;
      const bool valid = x < blk;
      const int b = i & 1;
      ok = mbar_wait(&e_full[b], (uint32_t)((i >> 1) & 1), kTfWaitNs, g.status);
      if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
      const int ea = eA_s[b][row];
      mbar_arrive(&e_empty[b]);
      ok = mbar_wait(&t_full, (uint32_t)(i & 1), kTfWaitNs, g.status);
      if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
      fence_after_sync();
      double2* dst = g.out + base * g.n_out + x;
      if (!STAGE && half >= n_chunks) {  // no chunk for this warp: release at once
        fence_before_sync();
        mbar_arrive(&t_empty);
      }
      // the 64-bit sums of chunk c (16 columns) of this thread's row
      auto sums = [&](int c, long long* S) {
#pragma unroll
        for (int j = 0; j < 16; ++j) S[j] = 0;
        int l = 0;
        for (; l + 1 < nslot - (nslot < 8 ? 1 : 0); l += 2) {  // pairs of single levels
          float v[32];
          tmem_ld16x2(tm + lane_base + (uint32_t)(l * NT + 16 * c), (uint32_t)NT, v);
          tf_add_pair<WIDE>(S, v, l);
        }
        for (; l < nslot; ++l) {  // what is left: a single level, the shared last one
          float v[16];
          tmem_ld16(tm + lane_base + (uint32_t)(l * NT + 16 * c), v);
          if (WIDE) tf_add_level_wide(S, v, l);
          else tf_add_level(S, v, l, l == nslot - 1 && nslot < 8);
        }
      };
      if (STAGE) {
        for (int c = half; c < n_chunks; c += 2) {
          long long S[16];
          sums(c, S);
#pragma unroll
          for (int j = 0; j < 16; ++j) Ss[(16 * c + j) * 128 + row] = S[j];
        }
        fence_before_sync();
        mbar_arrive(&t_empty);
      }
      for (int c = half; c < n_chunks; c += 2) {
        long long S[16];
        if (STAGE) {
#pragma unroll
          for (int j = 0; j < 16; ++j) S[j] = Ss[(16 * c + j) * 128 + row];
        } else {
          sums(c, S);
          if (c == last_c) {
            fence_before_sync();
            mbar_arrive(&t_empty);
          }
        }
        if (!valid) continue;
        const int n0 = ct * NT + 16 * c;  // first column of this chunk
        if (g.out_mode != kTfOutReal) {
          // columns 2m + c: component c of output slice m
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int n = n0 + j;
            if (n >= g.n_cols) break;
            const int m = n >> 1;
            const double re = i2d_scaled(S[j], ea + eB_s[n] - 52);
            const double im = i2d_scaled(S[j + 1], ea + eB_s[n + 1] - 52);
            dst[(long long)m * blk] = make_double2(re, im);
            if (g.out_mode == kTfOutMirror && g.n_out - 1 - m != m)
              dst[(long long)(g.n_out - 1 - m) * blk] = make_double2(re, dneg(im));
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + j;
            if (n >= g.n_cols) break;
            dst[(long long)(g.out_slice0 + n) * blk] = make_double2(i2d_scaled(S[j], ea + eB_s[n] - 52), 0.0);
          }
        }
      }
    }
    if (!ok) atomicExch(g.status, 2);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == kTfMmaWarp) tmem_dealloc(tm, 512);
}

}  // namespace

namespace {

// BF16 bits of the balanced digits of one scaled value, as tf_digit on the device.
void host_tf_digits(long long m, uint16_t* out) {
  const long long M = m + kTfBias;
  const long long t0 = M >= 0 ? (M >> 49) : -((-M + (1ll << 49) - 1) >> 49);  // floor(M / 2^49)
  auto bits = [](float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
  };
  out[0] = bits((float)t0);
  for (int s = 1; s < kOzDigits; ++s) {
    const int u = (int)((unsigned long long)M >> (49 - 7 * s)) & 127;
    out[s] = bits(std::ldexp((float)(u - 64), -7 * s));
  }
}

// Digits and exponents of the column operand B[n][k] = value(n, k), n < n_cols, k < K, in
// column tiles of NT.
template <typename F>
void tf_matrix(OzFused& f, int n_cols, int K, int NT, F value, std::vector<uint16_t>& dig, std::vector<int>& ex) {
  f.K = K;
  f.KS = (K + 15) / 16;
  f.n_cols = n_cols;
  f.NT = NT;
  f.n_ct = (n_cols + NT - 1) / NT;
  f.wide = f.K > 102;  // level sums may pass 2^22
  const size_t tile = (size_t)f.KS * kOzDigits * NT * 16;  // uint16 per column tile
  dig.assign(tile * f.n_ct, 0);
  ex.assign((size_t)NT * f.n_ct, 0);
  for (int n = 0; n < n_cols; ++n) {
    int mx = 0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, host_exp_field(value(n, k)));
    const int e = mx > 0 ? mx - 1022 : 0;
    ex[n] = e;
    const int ct = n / NT, nl = n % NT;
    for (int k = 0; k < K; ++k) {
      uint16_t d[kOzDigits];
      host_tf_digits(host_fixed56(value(n, k), e), d);
      const size_t at = ct * tile + (size_t)(k / 16) * kOzDigits * NT * 16 + umma::kmajor_offset(NT, nl, k % 16) / 2;
      for (int t = 0; t < kOzDigits; ++t) dig[at + (size_t)t * NT * 16] = d[t];
    }
  }
  // reductions up to 80 terms stage the epilogue's sums (two A stages); longer ones do not
  f.stage = f.KS <= kTfMaxKS;
  f.smem = (size_t)f.KS * kOzDigits * NT * 32 + (size_t)(f.stage ? 2 : 3) * kTfAStage +
           (f.stage ? (size_t)128 * NT * 8 : 0);
}

// Raises the instance's dynamic shared-memory limit, or (static_only) reports its static
// shared memory in *stat.
template <int KS, bool WIDE, bool STAGE>
cudaError_t tf_raise(size_t smem, bool static_only, size_t* stat) {
  if (static_only) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k_oz_transform<KS, WIDE, STAGE>);
    *stat = a.sharedSizeBytes;
    return e;
  }
  return raise_smem_limit(k_oz_transform<KS, WIDE, STAGE>, smem);
}
cudaError_t tf_raise_ks(int KS, size_t smem, bool static_only = false, size_t* stat = nullptr) {
  switch (KS) {
    case 1: return tf_raise<1, false, true>(smem, static_only, stat);
    case 2: return tf_raise<2, false, true>(smem, static_only, stat);
    case 3: return tf_raise<3, false, true>(smem, static_only, stat);
    case 4: return tf_raise<4, false, true>(smem, static_only, stat);
    case 5: return tf_raise<5, false, true>(smem, static_only, stat);
    case 6: return tf_raise<6, false, false>(smem, static_only, stat);
    case 7: return tf_raise<7, true, false>(smem, static_only, stat);
    default: return tf_raise<8, true, false>(smem, static_only, stat);
  }
}

void tf_launch(int KS, unsigned grid, size_t smem, cudaStream_t st, const TfArgs& a) {
  switch (KS) {
    case 1: k_oz_transform<1, false, true><<<grid, kTfThreads, smem, st>>>(a); break;
    case 2: k_oz_transform<2, false, true><<<grid, kTfThreads, smem, st>>>(a); break;
    case 3: k_oz_transform<3, false, true><<<grid, kTfThreads, smem, st>>>(a); break;
    case 4: k_oz_transform<4, false, true><<<grid, kTfThreads, smem, st>>>(a); break;
    case 5: k_oz_transform<5, false, true><<<grid, kTfThreads, smem, st>>>(a); break;
    case 6: k_oz_transform<6, false, false><<<grid, kTfThreads, smem, st>>>(a); break;
    case 7: k_oz_transform<7, true, false><<<grid, kTfThreads, smem, st>>>(a); break;
    default: k_oz_transform<8, true, false><<<grid, kTfThreads, smem, st>>>(a); break;
  }
}

}  // namespace

gw_status oz_fused_init(OzTransform& o, const HostPlan& h) {
  o.fw = OzFused{};
  o.fp = OzFused{};
  for (OzFused& f : o.fg) f = OzFused{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&o.n_sm, cudaDevAttrMultiProcessorCount, dev);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem_max <= 0) smem_max = 227 * 1024;
  const int N = h.n_tau, nh = (N + 1) / 2, nn = h.n_nu, nw = h.n_omega;
  std::vector<uint16_t> dig;
  std::vector<int> ex;
  auto upload = [&](OzFused& f) -> gw_status {
    // more than half of the SM's shared memory: one block per SM, so that no two blocks (of
    // this or another tensor-memory kernel on a concurrent stream) compete for the 512
    // tensor-memory columns each allocates
    f.smem = std::max(f.smem, (size_t)smem_max / 2 + 1024);
    size_t stat = 0;
    if (tf_raise_ks(f.KS, 0, true, &stat) != cudaSuccess) {
      set_last_error("querying the fused transform kernel failed");
      return GW_ERR_CUDA;
    }
    if (f.smem + stat > (size_t)smem_max) return GW_OK;  // does not fit: left to the other kernels
    if (cudaMalloc((void**)&f.d_B, dig.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc((void**)&f.d_e, ex.size() * sizeof(int)) != cudaSuccess) {
      set_last_error("device allocation for the fused transforms failed");
      return GW_ERR_OOM;
    }
    o.bytes += dig.size() * sizeof(uint16_t) + ex.size() * sizeof(int);
    if (cudaMemcpy(f.d_B, dig.data(), dig.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(f.d_e, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        tf_raise_ks(f.KS, f.smem) != cudaSuccess) {
      set_last_error("setting up the fused transforms failed");
      return GW_ERR_CUDA;
    }
    f.ready = true;
    return GW_OK;
  };
  gw_status s;
  // i nu -> tau of a real input: columns (Re, Im) of the nodes i < ceil(N/2) of the
  // mirror-symmetrised inverse, (T^-1_i + conj T^-1_{N-1-i}) / 2; the other nodes are
  // written as conjugates (W~(beta - tau) = conj W~(tau) for a real W~(i nu))
  if (2 * nh <= kTfMaxNT && nn <= 16 * kTfMaxKS) {
    const std::vector<double>& Ti = h.Tb_inv;  // [N][nn] complex
    tf_matrix(o.fw, 2 * nh, nn, (2 * nh + 15) / 16 * 16, [&](int n, int k) {
      const int i = n >> 1, c = n & 1;
      const size_t a = 2 * ((size_t)i * nn + k), b = 2 * ((size_t)(N - 1 - i) * nn + k);
      return c == 0 ? 0.5 * (Ti[a] + Ti[b]) : 0.5 * (Ti[a + 1] - Ti[b + 1]);
    }, dig, ex);
    if ((s = upload(o.fw)) != GW_OK) return s;
  }
  // tau -> i nu of a mirror-paired input: value 2i + c is component c of node i < ceil(N/2)
  if (nn <= kTfMaxNT && 2 * nh <= 16 * kTfMaxKS) {
    const std::vector<double>& Tm = h.Tb_mirror;  // [nn][nh] (a, b)
    tf_matrix(o.fp, nn, 2 * nh, (nn + 15) / 16 * 16,
              [&](int n, int k) { return Tm[2 * ((size_t)n * nh + (k >> 1)) + (k & 1)]; }, dig, ex);
    if ((s = upload(o.fp)) != GW_OK) return s;
  }
  // the same for the frequencies nu >= 0 only (sampled indices ascending: the first n_neg
  // are the negative ones)
  int n_neg = 0;
  while (n_neg < nn && h.nu_idx[n_neg] < 0) ++n_neg;
  bool ascending = true;
  for (int j = 1; j < nn; ++j) ascending = ascending && h.nu_idx[j] > h.nu_idx[j - 1];
  o.nu_nonneg0 = n_neg;
  if (ascending && nn - n_neg <= kTfMaxNT && 2 * nh <= 16 * kTfMaxKS && n_neg > 0) {
    const std::vector<double>& Tm = h.Tb_mirror;
    tf_matrix(o.fph, nn - n_neg, 2 * nh, (nn - n_neg + 15) / 16 * 16,
              [&](int n, int k) { return Tm[2 * ((size_t)(n_neg + n) * nh + (k >> 1)) + (k & 1)]; }, dig, ex);
    if ((s = upload(o.fph)) != GW_OK) return s;
  }
  // the general forms: complex input and output, value 2i + c of input slice i, column
  // 2m + c' of output slice m; B[2m + c'][2i + c] from T[m][i] = tr + i ti:
  // (c', c) = (0, 0): tr, (0, 1): -ti, (1, 0): ti, (1, 1): tr
  const std::vector<double>* mats[4] = {&h.Tf_fwd, &h.Tf_inv, &h.Tb_fwd, &h.Tb_inv};
  const int n_freq[2] = {nw, nn};
  for (int w = 0; w < 4; ++w) {
    const int fr = n_freq[w >> 1];
    const int n_in = (w & 1) ? fr : N, n_out = (w & 1) ? N : fr;
    if (2 * n_in > 16 * kTfMaxKSGeneral || 2 * n_out > kTfMaxCols) continue;
    const std::vector<double>& T = *mats[w];  // [n_out][n_in] complex
    tf_matrix(o.fg[w], 2 * n_out, 2 * n_in, 64, [&](int n, int k) {
      const size_t at = 2 * ((size_t)(n >> 1) * n_in + (k >> 1));
      const double tr = T[at], ti = T[at + 1];
      return (n & 1) == 0 ? ((k & 1) == 0 ? tr : -ti) : ((k & 1) == 0 ? ti : tr);
    }, dig, ex);
    if ((s = upload(o.fg[w])) != GW_OK) return s;
  }
  return GW_OK;
}

void oz_fused_free(OzTransform& o) {
  for (OzFused* f : {&o.fw, &o.fp, &o.fph, &o.fg[0], &o.fg[1], &o.fg[2], &o.fg[3]}) {
    if (f->d_B) cudaFree(f->d_B);
    if (f->d_e) cudaFree(f->d_e);
    *f = OzFused{};
  }
  if (o.d_tile_e_orb) cudaFree(o.d_tile_e_orb);
  if (o.d_tile_r0_orb) cudaFree(o.d_tile_r0_orb);
  o.d_tile_e_orb = o.d_tile_r0_orb = nullptr;
}

// One fused transform: `f` the column operand, `pb` the block kind (row tiles of o), the
// input form and where the columns go.
static gw_status tf_run(OzTransform& o, const OzFused& f, const DevEntry* d_ent, bool pb, const double2* in, int n_in,
                        int real_in, double2* out, int n_out, int out_mode, int* d_status, cudaStream_t st,
                        int out_slice0 = 0) {
  TfArgs a{};
  a.ent = d_ent;
  a.tile_e = pb ? o.d_tile_e : o.d_tile_e_orb;
  a.tile_r0 = pb ? o.d_tile_r0 : o.d_tile_r0_orb;
  a.n_rt = pb ? o.n_tiles : o.n_tiles_orb;
  a.n_ct = f.n_ct;
  a.pb = pb ? 1 : 0;
  a.in = in;
  a.n_in = n_in;
  a.K = f.K;
  a.real_in = real_in;
  a.out = out;
  a.n_out = n_out;
  a.out_mode = out_mode;
  a.out_slice0 = out_slice0;
  a.n_cols = f.n_cols;
  a.NT = f.NT;
  a.Bdig = f.d_B;
  a.eB = f.d_e;
  a.status = d_status;
  const int n_tiles = a.n_rt * a.n_ct;
  const unsigned grid = (unsigned)std::max(1, std::min(n_tiles, o.n_sm));
  {
    TimedLaunch tl_("k_oz_transform", st);
    tf_launch(f.KS, grid, f.smem, st, a);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("fused transform: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

gw_status oz_fused_run(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int structure, const double2* in,
                       double2* out, int* d_status, cudaStream_t st) {
  const bool w = structure == GW_IN_REAL;
  if (structure == (GW_IN_MIRROR | GW_OUT_NONNEG) && o.fph.ready)
    return tf_run(o, o.fph, d_ent, true, in, h.n_tau, 0, out, h.n_nu, kTfOutReal, d_status, st, o.nu_nonneg0);
  const OzFused& f = w ? o.fw : o.fp;
  if (!f.ready) {
    set_last_error("fused transform not planned");
    return GW_ERR_UNSUPPORTED;
  }
  return tf_run(o, f, d_ent, true, in, w ? h.n_nu : h.n_tau, w ? 1 : 0, out, w ? h.n_tau : h.n_nu,
                w ? kTfOutMirror : kTfOutReal, d_status, st);
}

bool oz_general_ready(const OzTransform& o, int fermion, int to_tau, bool pb) {
  return o.fg[(fermion ? 0 : 2) + (to_tau ? 1 : 0)].ready && (pb ? o.n_tiles > 0 : o.n_tiles_orb > 0);
}

gw_status oz_general_run(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int fermion, int to_tau, bool pb,
                         const double2* in, double2* out, int* d_status, cudaStream_t st) {
  const OzFused& f = o.fg[(fermion ? 0 : 2) + (to_tau ? 1 : 0)];
  const int fr = fermion ? h.n_omega : h.n_nu;
  return tf_run(o, f, d_ent, pb, in, to_tau ? fr : h.n_tau, 0, out, to_tau ? h.n_tau : fr, kTfOutComplex, d_status,
                st);
}

}  // namespace gw
